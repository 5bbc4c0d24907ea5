// rf_engine.h -- internal interface between the host orchestration
// (rf_api.cpp) and the CUDA kernels.  Plain C++ types only.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "realfast_gb300.h"

namespace rf {

// Gridding entry flags (low bits of GridEntry.cflags).
constexpr int ENT_CONJ = 1;  // contribute conj(R) (folded into the half plane)
constexpr int ENT_NEG = 2;   // checkerboard sign (-1)^(iu + iv) is -1

// One contribution of a (baseline, channel) visibility to a half-plane cell.
// bc = row c * nbl + b of the Stokes-I time series; cflags = (c << 2) | flags;
// row = the cell's v index iv mod N in its column; cell = the cell's global
// index (cells numbered by column, then row).
struct GridEntry {
  int32_t bc;
  int32_t cflags;
  int32_t row;
  int32_t cell;
};

// Device tables of a plan (all device pointers).
struct DevTables {
  const int32_t* delays;        // [ndm][nchan] integrations
  const int32_t* dt_list;       // [ndt]
  const int2* ranges;           // [nranges] cell-aligned entry ranges, one per gridding warp
  const int32_t* col_cell_ptr;  // [ncol + 1] first cell of each column
  const int32_t* cell_row;      // [ncells] row (iv mod N) of each cell
  const GridEntry* ent;         // [nent] sorted by (column, row)
  const int32_t* ongrid_chan;   // [nchan] on-grid baselines per channel
  const float2* twiddle;        // length-N FFT table (fft_twiddle_table(N)): [0, N) exp(+2 pi i m / N)
  // twiddle table of the column pass's sub-transforms, fft_twiddle_table(L)
  // with L = N / col_split(N) (the same table as `twiddle` when N <= 1024)
  const float2* twiddle_col;
  // runs of every imaged column: the column's cells at rows v1 + L v2 for one
  // v1 (cells sort by (v mod L, v div L) within a column, so a run is
  // consecutive); col_runs[col_run_ptr[col] + j] = (first cell << 4) | cells,
  // the first cell counted within the column
  const int32_t* col_run_ptr;   // [ncol + 1]
  const int32_t* col_runs;
  // per run j and sub-transform p = 1 .. R-1 (R = col_split(N) > 1): the
  // decimation-in-frequency twiddle w_N^(v1 p) of the run's row v1, at
  // col_run_tw[j (R - 1) + p - 1] (computed in FP64, rounded once)
  const float2* col_run_tw;
  // boxcar-resampled Stokes I per dt index s, phase-split: element (row, p, i)
  // at sdt_ptr[s] + row * dt * sdt_lp[s] + p * sdt_lp[s] + i holds
  // sum_{j < dt, i dt + p + j < nint} S[row][i dt + p + j]
  const unsigned long long* sdt_ptr;  // [ndt] device addresses (dt = 1: S itself)
  const int32_t* sdt_lp;              // [ndt] phase length ceil(nint_pad / dt)
};

// Group of consecutive output integrations of one (DM, dt) trial imaged
// together by the gridding/column-FFT kernel.
struct Group {
  int32_t d;
  int32_t s;
  int32_t t0;
  int32_t nimg;
  int32_t img0;  // index of the group's first image in the image list
  int32_t pad[3];
};

// One chunk of the fused imaging pass: nk consecutive images from image
// kbase of group g (absolute group index), whose column-FFT output shares one
// slot of the ring.
struct FusedChunk {
  int32_t g;
  int32_t kbase;
  int32_t nk;
  int32_t pad;
};

// Tensor map of a column-FFT output buffer T[slot][u][N] (as FP32 pairs) for
// the row pass's tile copies: nbox boxes of `rows` u rows each cover ncol.
struct TileMap {
  CUtensorMap map;
  int nbox;
  int rows;
};

// Launch options of the column and row passes when the waves of a search
// are overlapped (wave w + 1's column pass beside wave w's row pass, on two
// streams).  one_per_sm: the column pass asks for enough shared memory that
// a second column block no longer fits an SM, while a row block still does;
// items_per_block > 0: the row pass runs blocks of that many work items
// instead of one persistent block per slot, so that blocks of the two passes
// can take turns on an SM; priority (if set_priority): the launch's
// scheduling priority (lower values first).
struct PassLaunch {
  bool one_per_sm = false;
  int items_per_block = 0;
  bool set_priority = false;
  int priority = 0;
};

// Boxes of at most 256 rows (a multiple of 8) covering ncol rows.
inline void tile_boxes(int ncol, int* nbox, int* rows) {
  const int n0 = (ncol + 255) / 256;
  *rows = ((ncol + n0 - 1) / n0 + 7) / 8 * 8;  // whole swizzle atoms per box
  *nbox = (ncol + *rows - 1) / *rows;
}

// Statistics of one periodicity pair (DM trial d, fluctuation frequency k).
struct DevPeriodic {
  int32_t d, k, x, y;
  float amplitude, sigma, snr;
  int32_t pad;
};

// A candidate whose products are computed: trial (d, s, t') and pixel (x, y).
struct CandRef {
  int32_t d, s, t, x, y;
  int32_t pad[3];
};

// Twiddle table of a length-n FFT (n a power of two, 16..8192): entries
// [0, n) hold exp(+2 pi i m / n); when the transform has a second pass
// (n >= 64) entries n + (r / 2) 64 + 2 k + (r mod 2), r < P2, k < 32, hold
// that pass's twiddles exp(+2 pi i k r / (32 P2)), P2 = fft_pass2_radix(n)
// (the two r of a pair side by side, for 16-byte loads).  For n = 2048 a
// third section of the same layout, at n + 1024, holds
// exp(+2 pi i r (2k + 1) / 2048): the second-pass twiddles of the odd-pixel
// half of a row transform split into two length-1024 transforms, with the
// split's twiddle exp(+2 pi i r / 2048) folded in.  All are computed in FP64
// and rounded to FP32.
constexpr int fft_ilog2(int n) { return n <= 1 ? 0 : 1 + fft_ilog2(n >> 1); }
constexpr int fft_pass2_radix(int n) {
  // radix-E passes (E = 32, 16 for n = 16), the last of radix n / E^k
  return n < 64 ? 0 : (fft_ilog2(n) < 10 ? (1 << (fft_ilog2(n) - 5)) : 32);
}
constexpr int fft_twiddle_len(int n) { return n + 32 * fft_pass2_radix(n) + (n == 2048 ? 1024 : 0); }
// Fills out[0 .. fft_twiddle_len(n)).
void fft_twiddle_table(int n, float2* out);

// Cell of an off-grid (baseline, channel) in the per-row cell table.
constexpr int kOffGrid = -2147483647 - 1;

// Row-block partial statistics of one image (raw pixel units).  With the
// clipped noise, sum and sumsq hold the sums of d = J - mean0 and d^2 over
// the `kept` pixels J of the block with |d| <= clip sigmas (else zero).
struct StatPartial {
  double sum;
  double sumsq;
  float max;
  int32_t idx;  // y * N + x of max (lowest on ties)
  int32_t kept;
  int32_t pad;
};

// Clipping radius of the optional one-pass clipped noise, in units of the
// noise over all pixels.
constexpr double kClipSigmas = 5.0;

// Candidate record written on the device.
struct DevCand {
  int32_t d, s, t, x, y;
  float snr, peak, sigma;
};

// Per-image statistics written on the device (verification path).
struct DevStat {
  float peak, sigma, snr;
  int32_t x, y;
  int32_t pad;
  double mean;
  double weight;
};

struct SegmentGeom {
  int nint;       // integrations in this segment
  int nint_pad;   // row pitch of the Stokes-I buffer (elements)
  int nbl;
  int nchan;
  int npix;
  int ncol;       // half-plane columns imaged: 0 .. iu_max
  int ndm;
  int max_cells;  // largest number of occupied cells in one column
  int ncells;     // occupied cells of the half plane
  int nranges;    // gridding ranges
  bool partial;   // PARTIAL edge rule: a sample at or past nint is absent
  bool idx32;     // every sample index of every resampled series fits in 32 bits
  bool fp16;      // Stokes-I stored as half2
  // Row order of the column-FFT output T[slot][u][i]: with tsplit = R > 1,
  // index i = p L + k (L = N / R) holds image row y = R k + p (the column
  // pass's R sub-transforms of length L, one per residue p of y mod R, are
  // stored one after the other); tsplit <= 1: i = y.
  int tsplit;
};

// Sub-transforms per column in the batched column pass: N <= 1024 is one
// length-N transform; larger N are split R = N / 1024 ways along v (one
// radix-R decimation-in-frequency step folded into the gather of the
// column's cells), leaving R transforms of length 1024.
constexpr int col_split(int n) { return n >= 2048 ? n / 1024 : 1; }

// Complex values per thread of the row pass at N = 2048: 32 (64 threads per
// row pair, 256-thread blocks) or 16 (128 threads per row pair, 512-thread
// blocks: twice the warps in the same shared memory, at 64 registers a
// thread).  Both give the same images; 16 measured 36% slower on GB300
// (48.0 against 35.2 ms per 8134-image launch), so 32 is built.  The fused
// pass exists at 2048 only with 32.
#define RF_ROW_VALUES_2048 32

// ---------------------------------------------------------------- launchers
// All launchers return cudaSuccess or the launch error.

// Stokes-I ingest of integrations [t_begin, t_begin + nt) from `vis`
// ([nt][nbl][nchan][npol] complex64, already offset to t_begin) into the
// time-major buffer S[c * nbl + b][t].
cudaError_t launch_ingest(const float2* vis, int nt, int t_begin, int npol, const SegmentGeom& g, void* S,
                          cudaStream_t st);

// Subtract from every row of S its mean over the first nint integrations.
cudaError_t launch_mean_subtract(const SegmentGeom& g, void* S, cudaStream_t st);

// Boxcar resampling of S into the phase-split series of width dt (see
// DevTables::sdt_ptr) for the first nint integrations.
cudaError_t launch_resample(const SegmentGeom& g, const void* S, void* Sdt, int dt, int lp, cudaStream_t st);

// W of each listed image (img_info[i] = {d, s, t, 0}); n_on = on-grid
// (baseline, channel) pairs.
cudaError_t launch_weights(const int4* img_info, int nimg, bool partial, const SegmentGeom& g,
                           const DevTables& tb, double n_on, double* weight, cudaStream_t st);

// Gridding (pass A1) of groups [g_begin, g_begin + ngroups): the cell sums
// of every image, cellbuf[group - g_begin][cell][32 images].
cudaError_t launch_grid_cells(const SegmentGeom& g, const DevTables& tb, const Group* groups, int g_begin,
                              int ngroups, float2* cellbuf, cudaStream_t st);

// Column FFTs (pass A2) of the same groups from cellbuf; writes
// Tbuf[slot][col][y], slot = image index - img_base, the Parseval sums
// colsq[slot][col] (weighted sum of |H|^2 over the column) and
// mean0[slot] = Re H(u = 0, v = 0).
cudaError_t launch_colfft(const SegmentGeom& g, const DevTables& tb, const Group* groups, int g_begin,
                          int ngroups, int img_base, const float2* cellbuf, float2* Tbuf, float* colsq,
                          float* mean0, cudaStream_t st, const PassLaunch* pl = nullptr);

// Fused column + row pass (npix 1024 .. 4096) of the chunks [0, nchunks)
// of one wave (chunks[] on the device, groups indexed absolutely, cellbuf
// holding groups from g_begin): column FFTs into the ring Tring (ring slots
// of fused_chunk_images(N) images, tensor map tm), row FFTs and statistics
// into partials, Parseval sums into colsq/mean0 (slots relative to
// img_base).  counters: 1 + 2 nchunks ints (zeroed here).  err: set when a
// bounded wait gave up.
cudaError_t launch_image_fused(const SegmentGeom& g, const DevTables& tb, const Group* groups, int g_begin,
                               const FusedChunk* chunks, int nchunks, int img_base, const float2* cellbuf,
                               float2* Tring, int ring, const TileMap& tm, float* colsq, float* mean0,
                               StatPartial* partials, int* counters, int* err, cudaStream_t st);
// Images per chunk of the fused pass (0: no fused pass at this size).
int fused_chunk_images(int npix);

// Clipping window of each of `nimg` slots for the clipped noise, in raw
// pixel units (the image times 2W): clip[i] = {mean0[i], kClipSigmas *
// sigma over all pixels}, the sigma from the Parseval sums colsq.
cudaError_t launch_clip_window(const SegmentGeom& g, const float* colsq, const float* mean0, int nimg,
                               float2* clip, cudaStream_t st);

// Row C2R (pass B) + statistics of `nimg` images in slots [0, nimg) whose
// first image index is img_base.  Optionally writes the scaled images.
// With `clip` (per slot, from launch_clip_window) the partials also carry
// the kept-pixel sums of the clipped noise.
cudaError_t launch_rowfft_stats(const SegmentGeom& g, const DevTables& tb, const float2* Tbuf, int nimg,
                                int img_base, const double* weight, StatPartial* partials, float* images,
                                const TileMap* tm, int* err, cudaStream_t st, const float2* clip = nullptr,
                                const PassLaunch* pl = nullptr);

// Reduce row-block partials, compute sigma / snr, append candidates and
// (optionally) per-image stats for images [img_base, img_base + nimg).
// With `clip` the mean and sigma are those of the kept pixels, from the
// partials' sums around mean0.
cudaError_t launch_finalize(const SegmentGeom& g, const StatPartial* partials, const float* colsq,
                            const float* mean0, const int4* img_info, const double* weight, int nimg, int img_base,
                            double threshold, DevCand* cands, int* ncand, int cand_cap, DevStat* stats,
                            cudaStream_t st, bool clip = false);

// Buffers of the plain per-trial form (chunks of up to `cap` images).
struct PlainBuffers {
  const void* S;          // Stokes-I time series (as for the batched form)
  float2* R;              // [nbl * nchan][cap] dedispersed, resampled
  float2* grid;           // [cap][N][N/2 + 1] dense half planes
  float2* T;              // [cap][N/2][N] column-FFT output
  float* images;          // [cap][N][N]
  StatPartial* partials;  // [cap][partials per image] (row pass output, unused)
  const int4* ent;        // [nent] {bc, col, row, flags}
  int nent;
  int cap;
};

// One unfused launch set for images [img0, img0 + nk) = t' t0 .. t0+nk-1 of
// trial (d, s): dedisperse, grid (atomics), column FFTs, row FFTs writing the
// images, image statistics read back from HBM (a second read for the
// clipped noise with `clip`).
cudaError_t launch_plain_chunk(const SegmentGeom& g, const DevTables& tb, const PlainBuffers& pb, int d, int s,
                               int t0, int nk, int img0, const int4* img_info, const double* weight,
                               double threshold, DevCand* cands, int* ncand, int cand_cap, DevStat* stats,
                               cudaStream_t st, bool clip = false);

// Compile-time layout facts per image size, for host-side sizing.
struct ImageKernelShape {
  int images_per_group;   // B
  int cols_per_cta;       // C
  int threads_a;
  int smem_a;
  int warps_per_col;      // WPC: warps sharing one column's gridding (pass A)
  int rows_per_cta;       // RB (pass B)
  int partials_per_image; // partials written by pass B per image: N/2 row pairs x warps per transform
  int threads_b;
  int smem_b;
  int smem_a_per_cell;  // column pass: shared bytes per occupied cell of the largest column
  int smem_b_per_row;   // row pass: shared bytes per tile row (one per column imaged)
  bool tile_tma;        // row-pass tiles arrive by tensor copies (boxes, 1 KB alignment)
};
bool image_kernel_shape(int npix, ImageKernelShape* out);

// Streaming multiprocessors of the current device (cached per device: launch
// shapes are sized from it, and another GPU of the process may differ).
int sm_count();

// Sets the thread-local message returned by rf_last_error().
void set_last_error(const char* msg);

// Candidate products.  cellbc[c * nbl + b] = (iu, iv) or (kOffGrid, 0).
// spec/wch: [n][nchan] FP64 spectrum and w_c; spec_out: FP32 copy or NULL;
// spec_mom: [n][6] {mean, std, skew, excess kurtosis, w-mean, channels}.
cudaError_t launch_cand_spectrum(const SegmentGeom& g, const DevTables& tb, const int2* cellbc, const CandRef* refs,
                                 int n, double2* spec, double* wch, float2* spec_out, double* spec_mom,
                                 cudaStream_t st);
// out: [n][4] {mean, std, skew, excess kurtosis} of each image's npx pixels,
// in nslices slices per image (image_moment_slices); part: [n][nslices][4]
// scratch.
int image_moment_slices(int n, size_t npx);
cudaError_t launch_image_moments(const float* images, int n, size_t npx, int nslices, double* part, double* out,
                                 cudaStream_t st);

// Periodicity search.  Time transform of the dedispersed windows of nb DM
// trials (dms[j] indexes delays) into out[(2 j + q) nrows + row][kk].
cudaError_t launch_period_dft(const SegmentGeom& g, const void* S, const int* delays, const int* dms, int nb,
                              int L, const float2* twl, int kmin, int K, int kpad, float2* out, cudaStream_t st);
// Row pass over npairs (U, Q) image pairs: partials[j * N + y] = row maxima of I_U^2 + I_Q^2.
// tm (may be null): tensor map of Tbuf with boxes of one image's XB rows, for
// the tensor-copy tiles at N = 1024; err: set when a bounded tile wait gives up.
cudaError_t launch_rowfft_power(const SegmentGeom& g, const DevTables& tb, const float2* Tbuf, const int4* pairs,
                                int npairs, StatPartial* partials, const TileMap* tm, int* err, cudaStream_t st);
// Per pair: amplitude, sigma, snr, pixel; stats[pair_base + j]; candidates appended.
cudaError_t launch_finalize_power(const SegmentGeom& g, const StatPartial* partials, const float* colsq,
                                  const float* mean0, const int4* pairs, int npairs, int pair_base, double W,
                                  double threshold, DevPeriodic* stats, DevPeriodic* cands, int* ncand, int cand_cap,
                                  cudaStream_t st);

// One block waits, at most `polls` polls, on an mbarrier that nothing
// arrives at; *status = 1 when the wait gave up (it always should).
cudaError_t launch_wait_selftest(int polls, int* status, cudaStream_t st);

// ---------------------------------------------------------- host helpers --
// For the stream runtime (host code only).
struct PlanGeometry {
  int nbl, nchan, npol, max_nint, max_delay, device;
  bool host_only;
  std::vector<int> dt;
};
rf_status plan_geometry(const struct ::rf_plan* p, PlanGeometry* g);
// One search of nint integrations in which every (DM, dt) is limited to
// t' < span / dt besides the plan's edge rule (span 0: no limit).  Returns
// the candidates and, if stats is not NULL, every image's statistics.
rf_status search_span(struct ::rf_plan* p, const void* vis, int nint, int span, void* stream,
                      std::vector<rf_candidate>* cands, std::vector<rf_image_stat>* stats);

}  // namespace rf
