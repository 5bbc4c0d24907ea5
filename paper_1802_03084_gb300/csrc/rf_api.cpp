// rf_api.cpp -- the C ABI of include/realfast_gb300.h: plan construction
// (FP64 host tables), device buffers, and the orchestration of one segment
// search.  Compiled with -ffp-contract=off so the FP64 table arithmetic is
// plain IEEE double in the stated order.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "realfast_gb300.h"
#include "rf_engine.h"

using rf::DevCand;
using rf::DevStat;
using rf::GridEntry;
using rf::Group;
using rf::SegmentGeom;
using rf::StatPartial;

namespace {

thread_local std::string g_err;

rf_status fail(rf_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define RF_CUDA(call)                                                                            \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) return fail(RF_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                      \
  } while (0)

constexpr double kDispConst = 4.1488e-3;  // s GHz^2 per pc cm^-3 (Sec. 2.1 footnote)
constexpr double kCLight = 299792458.0;   // m/s
constexpr uint32_t kKnownFlags = RF_STORE_FP16 | RF_EDGE_PARTIAL | RF_MEAN_SUBTRACT | RF_NOISE_CLIPPED | RF_HOST_ONLY;
constexpr size_t kStageBytes = 256ull << 20;   // host->device chunk of raw visibilities
constexpr size_t kTBudgetBytes = 4096ull << 20;  // column-FFT scratch per wave
constexpr int kRangeEntries = 64;                // target entries per gridding warp
constexpr size_t kPeriodicBudgetBytes = 1ull << 30;  // transformed series per DM batch
constexpr size_t kPlainBudgetBytes = 4096ull << 20;  // plain form: intermediates of one chunk
constexpr int kDefaultRing = 3;                      // fused pass: chunk slots of the ring
constexpr int kOverlapRowItems = 16;                 // overlapped waves: work items per row-pass block

// Round half away from zero: sign(x) floor(|x| + 1/2).
inline double round_half_away(double x) { return x >= 0.0 ? std::floor(x + 0.5) : -std::floor(-x + 0.5); }

inline bool finite(double x) { return std::isfinite(x); }

struct Wave {
  int g_begin, g_end;
  int img_begin, img_end;
};

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Marks a plan busy for the duration of a call.
struct BusyGuard {
  std::atomic<int>* flag;
  bool owned = false;
  explicit BusyGuard(std::atomic<int>* f) : flag(f) {
    int expected = 0;
    owned = flag->compare_exchange_strong(expected, 1);
  }
  ~BusyGuard() {
    if (owned) flag->store(0);
  }
};

enum KernelKind {
  K_H2D = 0, K_INGEST, K_RESAMPLE, K_WEIGHTS, K_GRID_CELLS, K_GRID_COLFFT, K_ROWFFT_STATS, K_FINALIZE,
  K_PLAIN_TRIAL, K_MEAN_SUBTRACT, K_CLIP_WINDOW, K_IMAGE_FUSED, K_NKINDS
};
const char* const kKindNames[K_NKINDS] = {"h2d_copy",    "ingest",       "resample",
                                           "weights",     "grid_cells",   "grid_colfft",
                                           "rowfft_stats", "finalize",    "plain_trial_chunk",
                                           "mean_subtract", "clip_window", "image_fused"};

// Event-pair timing of every launch a plan issues while profiling is on.
struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> ev;  // pairs
  std::vector<int> kind;        // per pair
  size_t used = 0;
  int64_t launches[K_NKINDS] = {};
  double total_ms[K_NKINDS] = {};

  cudaEvent_t begin(int k, cudaStream_t st) {
    if (!on) return nullptr;
    if (used == kind.size()) {
      cudaEvent_t a, b;
      if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return nullptr;
      ev.push_back(a);
      ev.push_back(b);
      kind.push_back(k);
    }
    kind[used] = k;
    cudaEventRecord(ev[2 * used], st);
    return ev[2 * used + 1];
  }
  void end(cudaEvent_t e, cudaStream_t st) {
    if (!on || !e) return;
    cudaEventRecord(e, st);
    ++used;
  }
  // after the stream has synchronised
  void collect() {
    for (size_t i = 0; i < used; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]) == cudaSuccess) {
        launches[kind[i]]++;
        total_ms[kind[i]] += ms;
      } else {
        cudaGetLastError();
      }
    }
    used = 0;
  }
  // Hands the pairs [from, used) over to the caller (a captured graph) and
  // removes them from the pool.
  void take(size_t from, std::vector<cudaEvent_t>* evs, std::vector<int>* kinds) {
    for (size_t i = from; i < used; ++i) {
      evs->push_back(ev[2 * i]);
      evs->push_back(ev[2 * i + 1]);
      kinds->push_back(kind[i]);
    }
    ev.resize(2 * from);
    kind.resize(from);
    used = from;
  }
  void add_pairs(const std::vector<cudaEvent_t>& evs, const std::vector<int>& kinds) {
    for (size_t i = 0; i < kinds.size(); ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, evs[2 * i], evs[2 * i + 1]) == cudaSuccess) {
        launches[kinds[i]]++;
        total_ms[kinds[i]] += ms;
      } else {
        cudaGetLastError();
      }
    }
  }
  void reset() {
    used = 0;
    for (int k = 0; k < K_NKINDS; ++k) {
      launches[k] = 0;
      total_ms[k] = 0.0;
    }
  }
  void destroy() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
    ev.clear();
    kind.clear();
    used = 0;
  }
};

// Brackets one launch with the plan's profiler.
#define RF_TIMED(prof, kindv, st, call)            \
  do {                                             \
    cudaEvent_t e_end_ = (prof).begin(kindv, st);  \
    RF_CUDA(call);                                 \
    (prof).end(e_end_, st);                        \
  } while (0)

}  // namespace

struct rf_plan {
  // copy of the description
  int nant = 0, nchan = 0, npol = 0, npix = 0, ndm = 0, ndt = 0, max_nint = 0, device = 0;
  uint32_t flags = 0;
  double inttime = 0, cell = 0, threshold = 0;
  std::vector<double> ant_uvw, freq, dm;
  std::vector<int> dt;
  int form = RF_FORM_BATCHED;

  // host tables
  int nbl = 0;
  std::vector<double> bl_u, bl_v;
  std::vector<int32_t> delays;     // [ndm][nchan]
  std::vector<int32_t> max_delay;  // [ndm]
  std::vector<int32_t> iu, iv;     // [nbl][nchan]
  std::vector<uint8_t> ongrid;     // [nbl][nchan]
  std::vector<int32_t> col_ent_ptr, col_cell_ptr, cell_row;
  std::vector<int32_t> col_run_ptr, col_runs;  // runs of each column (see DevTables::col_runs)
  std::vector<float2> col_run_tw;              // their twiddles (see DevTables::col_run_tw)
  std::vector<int2> ranges;
  std::vector<int4> plain_ent;  // {bc, col, row, flags} for the plain form
  std::vector<GridEntry> ent;
  int n_cells = 0, max_cells = 0;
  std::vector<int32_t> ongrid_chan;
  int n_on = 0, iu_max = 0, iv_max = 0, ncol = 1, n_offgrid = 0;
  rf::ImageKernelShape shape{};

  // device state
  bool host_only = false;
  std::vector<void*> allocs;
  uint64_t device_bytes = 0;
  rf::DevTables tb{};
  void* d_S = nullptr;
  int nint_pad = 0;
  std::vector<void*> d_sdt;     // per dt index (dt = 1: d_S)
  std::vector<int32_t> sdt_lp;  // per dt index
  float2* d_T = nullptr;
  int slots_max = 0;
  StatPartial* d_partials = nullptr;
  double* d_weight = nullptr;
  int4* d_img_info = nullptr;
  Group* d_groups = nullptr;
  int img_cap = 0, group_cap = 0;
  DevCand* d_cands = nullptr;
  int* d_ncand = nullptr;
  DevStat* d_stats = nullptr;
  int2* d_cellbc = nullptr;     // [nchan * nbl] (iu, iv) per row, for candidate spectra
  int* d_err = nullptr;         // set by a kernel whose bounded wait gave up
  rf::TileMap tmap_T{};         // tensor map of d_T for the row pass (nbox 0: none)
  rf::TileMap tmap_P{};         // tensor map of d_T for the periodicity row pass (N = 1024)
  rf::TileMap tmap_H[2]{};      // tensor maps of the two halves of d_T (overlapped waves)
  float2* d_stage = nullptr;
  int stage_nint = 0;

  // image list of the last (nint, span) searched; span > 0 limits every
  // (DM, dt) to t' < span / dt (segments of a stream)
  int cached_nint = -1;
  int cached_span = 0;
  int t_span = 0;
  std::vector<int4> img_info;
  std::vector<Group> groups;
  std::vector<Wave> waves;
  int gslots_max = 0;           // groups per wave (cell buffer capacity)
  float2* d_cellbuf = nullptr;
  float* d_colsq = nullptr;     // [slots][ncol] Parseval sums
  float* d_mean0 = nullptr;     // [slots] Re H(0, 0)
  float2* d_clip = nullptr;     // [slots] clipping window (RF_NOISE_CLIPPED only)
  rf::PlainBuffers plain{};     // allocated on the first plain-form search

  // fused column + row pass (npix 1024 .. 4096): chunks of the image list,
  // the chunks of each wave, and the L2-resident ring of column-FFT output
  bool fused = false;           // RF_TUNE_FUSED (the autotuner turns it on where it wins)
  int ring = kDefaultRing;      // RF_TUNE_RING
  int chunk_images = 0;         // images per chunk (0: no fused pass at this size)
  std::vector<rf::FusedChunk> chunks;
  std::vector<int2> wave_chunks;  // per wave: [first, last) chunk
  rf::FusedChunk* d_chunks = nullptr;
  int* d_fcount = nullptr;      // 1 + 2 x (most chunks of a wave) counters
  int fcount_cap = 0;
  float2* d_Tring = nullptr;
  int ring_alloc = 0;
  rf::TileMap tmap_ring{};

  // overlapped waves (RF_TUNE_OVERLAP): waves of at most half the slots
  // alternate between the halves of the scratch; wave w + 1's gridding and
  // column pass run on the caller's stream beside wave w's row pass and
  // finalize on ostream.  oev: column pass done [2], row pass and finalize
  // done [2] (per half), and the join back to the caller's stream.
  bool overlap = false;
  bool waves_overlap = false;   // the current wave list was built for it
  cudaStream_t ostream = nullptr;
  cudaEvent_t oev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};

  // CUDA graph of the batched wave loop for the current image list
  bool use_graphs = true;
  bool wide_index = false;      // RF_TUNE_WIDE_INDEX: 64-bit gridding sample offsets always
  bool graph_pending = false;  // a replay with profiling events awaits collection
  struct GraphCache {
    bool valid = false;
    int nint = -1;
    bool stats = false;
    bool prof = false;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> ev;  // profiler event pairs captured in the graph
    std::vector<int> kind;
  } graph;
  cudaStream_t gstream = nullptr;  // private stream: capture and replay
  cudaEvent_t join[2] = {nullptr, nullptr};

  void drop_graph() {
    if (graph.exec) cudaGraphExecDestroy(graph.exec);
    for (cudaEvent_t e : graph.ev) cudaEventDestroy(e);
    graph = GraphCache();
  }

  std::atomic<int> busy{0};
  Profiler prof;

  template <class T>
  rf_status dalloc(T** p, size_t count) {
    void* q = nullptr;
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(RF_ERR_NO_MEMORY, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    allocs.push_back(q);
    device_bytes += bytes;
    *p = static_cast<T*>(q);
    return RF_OK;
  }

  void dfree(void* q) {
    for (size_t i = 0; i < allocs.size(); ++i)
      if (allocs[i] == q) {
        cudaFree(q);
        allocs.erase(allocs.begin() + i);
        return;
      }
  }

  ~rf_plan() {
    if (!allocs.empty() || !prof.ev.empty() || gstream || ostream) {
      DeviceGuard dg(device);
      drop_graph();
      if (gstream) cudaStreamDestroy(gstream);
      for (cudaEvent_t e : join)
        if (e) cudaEventDestroy(e);
      if (ostream) cudaStreamDestroy(ostream);
      for (cudaEvent_t e : oev)
        if (e) cudaEventDestroy(e);
      for (void* p : allocs) cudaFree(p);
      prof.destroy();
    }
  }
};

namespace {

int n_times_span(const rf_plan* p, int nint, int d, int s, int t_span) {
  const int dt = p->dt[s];
  int n;
  if (p->flags & RF_EDGE_PARTIAL) {
    n = nint / dt;
  } else {
    const int span = nint - p->max_delay[d];
    n = span > 0 ? span / dt : 0;
  }
  return t_span > 0 ? std::min(n, t_span / dt) : n;
}

int n_times(const rf_plan* p, int nint, int d, int s) { return n_times_span(p, nint, d, s, p->t_span); }

int64_t count_images(const rf_plan* p, int nint) {
  int64_t n = 0;
  for (int d = 0; d < p->ndm; ++d)
    for (int s = 0; s < p->ndt; ++s) n += n_times(p, nint, d, s);
  return n;
}

rf_status validate(const rf_plan_desc* d) {
  if (!d) return fail(RF_ERR_INVALID_ARG, "desc is NULL");
  if (d->nant < 2 || d->nant > 4096) return fail(RF_ERR_INVALID_ARG, "nant %d out of [2, 4096]", d->nant);
  if (!d->ant_uvw_m) return fail(RF_ERR_INVALID_ARG, "ant_uvw_m is NULL");
  if (d->nchan < 1 || d->nchan > 65536) return fail(RF_ERR_INVALID_ARG, "nchan %d out of [1, 65536]", d->nchan);
  if (!d->freq_hz) return fail(RF_ERR_INVALID_ARG, "freq_hz is NULL");
  if (d->npol != 1 && d->npol != 2) return fail(RF_ERR_INVALID_ARG, "npol must be 1 or 2");
  if (!(d->inttime_s > 0.0) || !finite(d->inttime_s)) return fail(RF_ERR_INVALID_ARG, "inttime_s must be > 0");
  if (d->npix < 16 || d->npix > 8192 || (d->npix & (d->npix - 1)))
    return fail(RF_ERR_INVALID_ARG, "npix %d is not a power of two in [16, 8192]", d->npix);
  if (!(d->cell_rad > 0.0) || !finite(d->cell_rad)) return fail(RF_ERR_INVALID_ARG, "cell_rad must be > 0");
  if (d->ndm < 1 || !d->dm_list) return fail(RF_ERR_INVALID_ARG, "need ndm >= 1 and dm_list");
  if (d->ndt < 1 || d->ndt > 64 || !d->dt_list) return fail(RF_ERR_INVALID_ARG, "need 1 <= ndt <= 64 and dt_list");
  if (!(d->threshold_sigma > 0.0) || !finite(d->threshold_sigma))
    return fail(RF_ERR_INVALID_ARG, "threshold_sigma must be > 0");
  if (d->flags & ~kKnownFlags) return fail(RF_ERR_INVALID_ARG, "unknown flag bits 0x%x", d->flags & ~kKnownFlags);
  if (d->max_nint < 1 || d->max_nint > (1 << 24)) return fail(RF_ERR_INVALID_ARG, "max_nint %d out of range", d->max_nint);
  for (int i = 0; i < 3 * d->nant; ++i)
    if (!finite(d->ant_uvw_m[i])) return fail(RF_ERR_INVALID_ARG, "ant_uvw_m[%d] is not finite", i);
  for (int c = 0; c < d->nchan; ++c)
    if (!(d->freq_hz[c] > 0.0) || !finite(d->freq_hz[c])) return fail(RF_ERR_INVALID_ARG, "freq_hz[%d] must be > 0", c);
  for (int i = 0; i < d->ndm; ++i)
    if (!(d->dm_list[i] >= 0.0) || !finite(d->dm_list[i])) return fail(RF_ERR_INVALID_ARG, "dm_list[%d] must be >= 0", i);
  for (int i = 0; i < d->ndt; ++i)
    if (d->dt_list[i] < 1 || d->dt_list[i] > 1024) return fail(RF_ERR_INVALID_ARG, "dt_list[%d] out of [1, 1024]", i);
  const int64_t nbl = (int64_t)d->nant * (d->nant - 1) / 2;
  if (nbl * d->nchan > (1ll << 28)) return fail(RF_ERR_INVALID_ARG, "nbl * nchan too large");
  return RF_OK;
}

// Host tables in FP64 (Sec. 2.1 dispersion law; Sec. 2.2 baselines).
rf_status build_tables(rf_plan* p) {
  const int nant = p->nant, nchan = p->nchan, N = p->npix;
  p->nbl = nant * (nant - 1) / 2;
  const int nbl = p->nbl;
  p->bl_u.resize(nbl);
  p->bl_v.resize(nbl);
  int b = 0;
  for (int i = 0; i < nant; ++i)
    for (int j = i + 1; j < nant; ++j, ++b) {
      p->bl_u[b] = p->ant_uvw[3 * j + 0] - p->ant_uvw[3 * i + 0];
      p->bl_v[b] = p->ant_uvw[3 * j + 1] - p->ant_uvw[3 * i + 1];
    }

  // delay[d][c] = floor(((K dm) (1/(f f) - 1/(ft ft))) / tint + 1/2), f in GHz
  double ftop_hz = p->freq[0];
  for (double f : p->freq) ftop_hz = std::max(ftop_hz, f);
  const double ft = ftop_hz * 1e-9;
  std::vector<double> dinv(nchan);
  for (int c = 0; c < nchan; ++c) {
    const double f = p->freq[c] * 1e-9;
    dinv[c] = (1.0 / (f * f)) - (1.0 / (ft * ft));
  }
  p->delays.assign((size_t)p->ndm * nchan, 0);
  p->max_delay.assign(p->ndm, 0);
  for (int d = 0; d < p->ndm; ++d) {
    const double kd = kDispConst * p->dm[d];
    int mx = 0;
    for (int c = 0; c < nchan; ++c) {
      const double x = (kd * dinv[c]) / p->inttime;
      const double r = std::floor(x + 0.5);
      if (!(r >= 0.0) || r > (double)(1 << 26)) return fail(RF_ERR_INVALID_ARG, "delay of DM %g out of range", p->dm[d]);
      const int v = (int)r;
      p->delays[(size_t)d * nchan + c] = v;
      mx = std::max(mx, v);
    }
    p->max_delay[d] = mx;
  }

  // nearest cells: i = round_half_away((u_m (f / c)) (N cell))
  const double fov = (double)N * p->cell;
  p->iu.assign((size_t)nbl * nchan, 0);
  p->iv.assign((size_t)nbl * nchan, 0);
  p->ongrid.assign((size_t)nbl * nchan, 0);
  p->ongrid_chan.assign(nchan, 0);
  const int half = N / 2;
  p->n_on = 0;
  p->n_offgrid = 0;
  p->iu_max = 0;
  p->iv_max = 0;
  for (int bb = 0; bb < nbl; ++bb)
    for (int c = 0; c < nchan; ++c) {
      const double s = p->freq[c] / kCLight;
      const double xu = (p->bl_u[bb] * s) * fov;
      const double xv = (p->bl_v[bb] * s) * fov;
      const double ru = round_half_away(xu), rv = round_half_away(xv);
      const size_t k = (size_t)bb * nchan + c;
      const bool on = std::fabs(ru) < half && std::fabs(rv) < half;
      p->iu[k] = on ? (int)ru : (int)std::max(-2147483647.0, std::min(2147483647.0, ru));
      p->iv[k] = on ? (int)rv : (int)std::max(-2147483647.0, std::min(2147483647.0, rv));
      p->ongrid[k] = on ? 1 : 0;
      if (on) {
        p->n_on++;
        p->ongrid_chan[c]++;
        p->iu_max = std::max(p->iu_max, std::abs((int)ru));
        p->iv_max = std::max(p->iv_max, std::abs((int)rv));
      } else {
        p->n_offgrid++;
      }
    }

  // half-plane columns 0..iu_max: entries sorted by (col, row, bc, flags)
  struct E {
    int col, row, bc, flags;
  };
  std::vector<E> es;
  es.reserve((size_t)p->n_on + nbl);
  auto mod = [N](int x) { return ((x % N) + N) % N; };
  for (int bb = 0; bb < nbl; ++bb)
    for (int c = 0; c < nchan; ++c) {
      const size_t k = (size_t)bb * nchan + c;
      if (!p->ongrid[k]) continue;
      const int u = p->iu[k], v = p->iv[k];
      const int neg = ((u + v) & 1) ? rf::ENT_NEG : 0;
      const int bc = c * nbl + bb;
      if (u > 0) {
        es.push_back({u, mod(v), bc, neg});
      } else if (u < 0) {
        es.push_back({-u, mod(-v), bc, rf::ENT_CONJ | neg});
      } else {
        es.push_back({0, mod(v), bc, neg});
        es.push_back({0, mod(-v), bc, rf::ENT_CONJ | neg});
      }
    }
  // Within a column, rows sort by (v mod L, v div L), L = N / col_split(N):
  // the batched column pass finds the rows that share v mod L (combined by
  // its decimation-in-frequency gather) next to each other.  For N <= 1024,
  // L = N and this is plain row order.
  const int Lc = N / rf::col_split(N);
  std::sort(es.begin(), es.end(), [Lc](const E& a, const E& b2) {
    if (a.col != b2.col) return a.col < b2.col;
    const int ka = a.row % Lc, kb = b2.row % Lc;
    if (ka != kb) return ka < kb;
    if (a.row != b2.row) return a.row < b2.row;
    if (a.bc != b2.bc) return a.bc < b2.bc;
    return a.flags < b2.flags;
  });
  p->ncol = p->n_on > 0 ? p->iu_max + 1 : 1;
  if (!rf::image_kernel_shape(N, &p->shape)) return fail(RF_ERR_INVALID_ARG, "npix %d has no kernel", N);
  p->plain_ent.clear();
  p->plain_ent.reserve(es.size());
  for (const E& e : es) p->plain_ent.push_back(make_int4(e.bc, e.col, e.row, e.flags));
  p->ent.clear();
  p->ent.reserve(es.size());
  p->col_ent_ptr.assign(p->ncol + 1, 0);
  p->col_cell_ptr.assign(p->ncol + 1, 0);
  p->cell_row.clear();
  p->n_cells = 0;
  p->max_cells = 0;
  std::vector<int> cell_start;  // entry index where each cell begins
  size_t i = 0;
  for (int col = 0; col < p->ncol; ++col) {
    p->col_ent_ptr[col] = (int)p->ent.size();
    p->col_cell_ptr[col] = p->n_cells;
    int prev_row = -1;
    int local = -1;
    while (i < es.size() && es[i].col == col) {
      if (es[i].row != prev_row) {
        cell_start.push_back((int)p->ent.size());
        prev_row = es[i].row;
        p->cell_row.push_back(es[i].row);
        p->n_cells++;
        ++local;
      }
      const int c = es[i].bc / nbl;
      p->ent.push_back({es[i].bc, (c << 2) | es[i].flags, es[i].row, p->n_cells - 1});
      ++i;
    }
    p->max_cells = std::max(p->max_cells, local + 1);
  }
  p->col_ent_ptr[p->ncol] = (int)p->ent.size();
  p->col_cell_ptr[p->ncol] = p->n_cells;
  // runs of each column for the column pass's scatter
  p->col_run_ptr.assign(p->ncol + 1, 0);
  p->col_runs.clear();
  for (int col = 0; col < p->ncol; ++col) {
    const int c0 = p->col_cell_ptr[col], c1 = p->col_cell_ptr[col + 1];
    p->col_run_ptr[col] = (int)p->col_runs.size();
    for (int c = c0; c < c1;) {
      const int v1 = p->cell_row[c] % Lc;
      int n = 1;
      while (c + n < c1 && p->cell_row[c + n] % Lc == v1) ++n;
      p->col_runs.push_back(((c - c0) << 4) | n);
      c += n;
    }
  }
  p->col_run_ptr[p->ncol] = (int)p->col_runs.size();
  {
    // w_N^(v1 p) of every run for p = 1 .. R-1, FP64 and rounded once (the
    // same values as the length-N twiddle table)
    const int R = rf::col_split(N);
    p->col_run_tw.assign(p->col_runs.size() * (size_t)std::max(R - 1, 1), make_float2(0.f, 0.f));
    const double two_pi = 6.283185307179586476925286766559;
    for (int col = 0; col < p->ncol; ++col)
      for (int j = p->col_run_ptr[col]; j < p->col_run_ptr[col + 1]; ++j) {
        const int v1 = p->cell_row[p->col_cell_ptr[col] + (p->col_runs[j] >> 4)] % Lc;
        for (int q = 1; q < R; ++q) {
          const double a = two_pi * (double)((v1 * q) % N) / (double)N;
          p->col_run_tw[(size_t)j * (R - 1) + q - 1] = make_float2((float)std::cos(a), (float)std::sin(a));
        }
      }
  }
  cell_start.push_back((int)p->ent.size());
  // Cell-aligned entry ranges of about kRangeEntries entries (a range holds
  // whole cells; a cell with more entries is a range of its own).
  p->ranges.clear();
  {
    size_t ci = 0;
    while (ci + 1 < cell_start.size()) {
      const int eb = cell_start[ci];
      size_t cj = ci + 1;
      while (cj + 1 < cell_start.size() && cell_start[cj + 1] - eb <= kRangeEntries) ++cj;
      p->ranges.push_back(make_int2(eb, cell_start[cj]));
      ci = cj;
    }
  }
  // The column pass stages the cells of one column, and the row pass one tile
  // of ncol rows, in a block's shared memory (at most 227 KB on sm_103a, less
  // up to 1 KB of the kernels' static shared memory).
  {
    const long limit = 227l * 1024 - 1024;
    const rf::ImageKernelShape& sh = p->shape;
    const long smem_a = (long)sh.smem_a + (long)p->max_cells * sh.smem_a_per_cell;
    int tile_rows = p->ncol;
    if (sh.tile_tma) {
      int nbox = 0, rows = 0;
      rf::tile_boxes(p->ncol, &nbox, &rows);
      tile_rows = nbox * rows;
    }
    const long smem_b = (long)sh.smem_b + (sh.tile_tma ? 1024 : 0) + (long)tile_rows * sh.smem_b_per_row;
    if (smem_a > limit)
      return fail(RF_ERR_INVALID_ARG,
                  "a uv column holds %d occupied cells; the column pass fits at most %ld at npix %d "
                  "(a coarser cell or a smaller npix spreads fewer cells per column)",
                  p->max_cells, (limit - sh.smem_a) / sh.smem_a_per_cell, N);
    if (smem_b > limit)
      return fail(RF_ERR_INVALID_ARG, "%d uv columns do not fit the row pass's shared memory at npix %d", p->ncol, N);
  }
  return RF_OK;
}

// Whether waves can be overlapped: asked for, two halves of the scratch hold
// a group each, and neither the fused pass nor the clipped noise (whose
// window buffer is per slot of the whole scratch) is in use.
bool overlap_possible(const rf_plan* p) {
  return p->overlap && !p->fused && !(p->flags & RF_NOISE_CLIPPED) &&
         p->slots_max / 2 >= p->shape.images_per_group;
}

// Image and group lists for a segment of nint integrations, in (d, s, t') order.
void build_lists(rf_plan* p, int nint) {
  const int B = p->shape.images_per_group;
  p->img_info.clear();
  p->groups.clear();
  p->waves.clear();
  for (int d = 0; d < p->ndm; ++d)
    for (int s = 0; s < p->ndt; ++s) {
      const int nt = n_times(p, nint, d, s);
      for (int t0 = 0; t0 < nt; t0 += B) {
        Group g{};
        g.d = d;
        g.s = s;
        g.t0 = t0;
        g.nimg = std::min(B, nt - t0);
        g.img0 = (int)p->img_info.size();
        p->groups.push_back(g);
        for (int k = 0; k < g.nimg; ++k) p->img_info.push_back(make_int4(d, s, t0 + k, 0));
      }
    }
  // overlapped waves take half the slots each (see run_waves)
  p->waves_overlap = overlap_possible(p);
  const int cap = p->waves_overlap ? p->slots_max / 2 : p->slots_max;
  Wave w{0, 0, 0, 0};
  for (int gi = 0; gi < (int)p->groups.size(); ++gi) {
    const Group& g = p->groups[gi];
    if (g.img0 + g.nimg - w.img_begin > cap || gi - w.g_begin >= p->gslots_max) {
      w.g_end = gi;
      w.img_end = g.img0;
      p->waves.push_back(w);
      w = Wave{gi, gi, g.img0, g.img0};
    }
  }
  w.g_end = (int)p->groups.size();
  w.img_end = (int)p->img_info.size();
  if (w.img_end > w.img_begin) p->waves.push_back(w);
  // chunks of the fused pass: each group's images in runs of chunk_images
  p->chunks.clear();
  p->wave_chunks.clear();
  if (p->chunk_images > 0) {
    for (const Wave& wv : p->waves) {
      const int c0 = (int)p->chunks.size();
      for (int gi = wv.g_begin; gi < wv.g_end; ++gi)
        for (int k = 0; k < p->groups[gi].nimg; k += p->chunk_images)
          p->chunks.push_back({gi, k, std::min(p->chunk_images, p->groups[gi].nimg - k), 0});
      p->wave_chunks.push_back(make_int2(c0, (int)p->chunks.size()));
    }
  }
  p->cached_nint = nint;
  p->cached_span = p->t_span;
  p->drop_graph();
}

// Whether the search's waves take the fused column + row pass.
bool use_fused(const rf_plan* p) {
  return p->fused && p->chunk_images > 0 && p->tmap_ring.nbox > 0 && !(p->flags & RF_NOISE_CLIPPED);
}

// cuTensorMapEncodeTiled from the driver, looked up once.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

// Tensor map of the column-FFT output d_T ([slots][ncol][N] complex, seen as
// FP32 pairs) for the row pass's tile copies, N >= 1024: the box is one
// work item's 2 XB rows (XB 16-byte chunks) by `rows` columns u, swizzled so
// that chunk c of column u lands at c ^ ((u >> sh) & (XB - 1)).  Where the
// encoder is unavailable the row pass copies with cp.async (nbox = 0).
// Tensor map of T ([slot][u][N complex]) whose boxes hold `trows` T rows of
// `rows` u rows; box rows of 128, 64 or 32 bytes are swizzled in that mode.
// The search's row pass takes the 2 XB rows of a work item (trows = 2 XB),
// the periodicity row pass the XB rows of one image (trows = XB).
void encode_tile_map(rf_plan* p, rf::TileMap& tm, float2* base, int slots, int trows) {
  tm.nbox = 0;
  const int N = p->npix;
  if (N < 1024 || !base || slots <= 0) return;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return;
  int nbox, rows;
  rf::tile_boxes(p->ncol, &nbox, &rows);
  const int row_bytes = trows * 8;
  const cuuint64_t dims[3] = {(cuuint64_t)2 * N, (cuuint64_t)p->ncol, (cuuint64_t)slots};
  const cuuint64_t strides[2] = {(cuuint64_t)N * 8, (cuuint64_t)p->ncol * N * 8};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * trows), (cuuint32_t)rows, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUtensorMapSwizzle sw = row_bytes == 128  ? CU_TENSOR_MAP_SWIZZLE_128B
                                : row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                : row_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                                  : CU_TENSOR_MAP_SWIZZLE_NONE;
  const CUresult r = enc(&tm.map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r == CUDA_SUCCESS) {
    tm.nbox = nbox;
    tm.rows = rows;
  }
}

// (Re)allocate the per-wave scratch for `slots` images (clamped to
// [images_per_group, 32768]: images per wave ride on gridDim.y).
rf_status alloc_wave_scratch(rf_plan* p, int slots) {
  const int B = p->shape.images_per_group;
  slots = std::max(std::min(slots, 32768), B);
  const size_t per_slot = (size_t)p->ncol * p->npix;
  const int nrb = p->shape.partials_per_image;
  p->tmap_T.nbox = 0;  // the maps describe d_T, about to be freed
  p->tmap_P.nbox = 0;
  p->tmap_H[0].nbox = p->tmap_H[1].nbox = 0;
  if (p->d_T) {
    p->device_bytes -= (uint64_t)p->slots_max * per_slot * sizeof(float2);
    p->dfree(p->d_T);
    p->d_T = nullptr;
  }
  if (p->d_partials) {
    p->device_bytes -= (uint64_t)p->slots_max * nrb * sizeof(StatPartial);
    p->dfree(p->d_partials);
    p->d_partials = nullptr;
  }
  if (p->d_cellbuf) {
    p->device_bytes -= (uint64_t)p->gslots_max * p->n_cells * 32 * sizeof(float2);
    p->dfree(p->d_cellbuf);
    p->d_cellbuf = nullptr;
  }
  if (p->d_colsq) {
    p->device_bytes -= (uint64_t)p->slots_max * (p->ncol + 1) * sizeof(float);
    p->dfree(p->d_colsq);
    p->dfree(p->d_mean0);
    p->d_colsq = p->d_mean0 = nullptr;
  }
  if (p->d_clip) {
    p->device_bytes -= (uint64_t)p->slots_max * sizeof(float2);
    p->dfree(p->d_clip);
    p->d_clip = nullptr;
  }
  p->slots_max = slots;
  p->gslots_max = std::max(2 * ((slots + B - 1) / B), 1);
  p->cached_nint = -1;
  p->drop_graph();
  rf_status s;
  if ((s = p->dalloc(&p->d_T, (size_t)slots * per_slot)) != RF_OK) return s;
  if ((s = p->dalloc(&p->d_partials, (size_t)slots * nrb)) != RF_OK) return s;
  if ((s = p->dalloc(&p->d_cellbuf, (size_t)p->gslots_max * std::max(p->n_cells, 1) * 32)) != RF_OK) return s;
  if ((s = p->dalloc(&p->d_colsq, (size_t)slots * p->ncol)) != RF_OK) return s;
  if ((s = p->dalloc(&p->d_mean0, (size_t)slots)) != RF_OK) return s;
  if ((p->flags & RF_NOISE_CLIPPED) && (s = p->dalloc(&p->d_clip, (size_t)slots)) != RF_OK) return s;
  const int xb = std::min(256 / (p->npix / 32), p->npix / 2);  // row pairs of a row-pass work item
  encode_tile_map(p, p->tmap_T, p->d_T, p->slots_max, 2 * xb);
  // the halves of d_T, each a wave's scratch when waves are overlapped
  const int half = p->slots_max / 2;
  if (half >= B) {
    encode_tile_map(p, p->tmap_H[0], p->d_T, half, 2 * xb);
    encode_tile_map(p, p->tmap_H[1], p->d_T + (size_t)half * per_slot, half, 2 * xb);
  }
  // the periodicity row pass's tensor-copy tiles (one image's XB rows), at
  // N = 1024, where its transforms fit one warp
  if (p->npix == 1024) encode_tile_map(p, p->tmap_P, p->d_T, p->slots_max, xb);
  // fused pass: counters for the most chunks a wave can hold
  if (p->chunk_images > 0) {
    const int cap = 1 + 2 * p->gslots_max * ((p->shape.images_per_group + p->chunk_images - 1) / p->chunk_images);
    if (p->d_fcount) {
      p->device_bytes -= (uint64_t)p->fcount_cap * sizeof(int);
      p->dfree(p->d_fcount);
      p->d_fcount = nullptr;
    }
    if ((s = p->dalloc(&p->d_fcount, (size_t)cap)) != RF_OK) return s;
    p->fcount_cap = cap;
  }
  return RF_OK;
}

// (Re)allocate the fused pass's ring of `ring` chunk slots and its tensor map.
rf_status alloc_ring(rf_plan* p, int ring) {
  if (p->chunk_images <= 0) return RF_OK;
  const size_t per_ring = (size_t)p->chunk_images * p->ncol * p->npix;
  p->tmap_ring.nbox = 0;
  p->drop_graph();
  if (p->d_Tring) {
    p->device_bytes -= (uint64_t)p->ring_alloc * per_ring * sizeof(float2);
    p->dfree(p->d_Tring);
    p->d_Tring = nullptr;
  }
  rf_status s = p->dalloc(&p->d_Tring, (size_t)ring * per_ring);
  if (s != RF_OK) return s;
  p->ring = p->ring_alloc = ring;
  encode_tile_map(p, p->tmap_ring, p->d_Tring, ring * p->chunk_images,
                  2 * std::min(256 / (p->npix / 32), p->npix / 2));
  return RF_OK;
}

// Device bytes alloc_device will allocate for a plan whose host tables are
// built, with column-FFT scratch for `slots` images (0 = the default
// budget).  Mirrors alloc_device and alloc_wave_scratch.
uint64_t estimate_device_bytes(const rf_plan* p, int slots) {
  const size_t N = p->npix;
  auto r = [](size_t n, size_t sz) { return (uint64_t)std::max<size_t>(n, 1) * sz; };
  uint64_t b = 0;
  b += r(p->delays.size(), 4) + r(p->dt.size(), 4) + r(p->ranges.size(), 8) + r(p->col_cell_ptr.size(), 4) +
       r(p->cell_row.size(), 4) + r(p->col_run_ptr.size(), 4) + r(p->col_runs.size(), 4) + r(p->col_run_tw.size(), 8) + r(p->ent.size(), sizeof(GridEntry)) + r(p->ongrid_chan.size(), 4) + r(rf::fft_twiddle_len((int)N), 8);
  if (rf::col_split((int)N) > 1) b += r(rf::fft_twiddle_len((int)N / rf::col_split((int)N)), 8);
  const size_t nint_pad = (p->max_nint + 31) / 32 * 32;
  const size_t esz = (p->flags & RF_STORE_FP16) ? 4 : 8;
  const size_t rows = (size_t)p->nbl * p->nchan;
  b += r(rows * nint_pad, esz);
  std::vector<int> seen;
  for (int dt : p->dt) {
    if (dt == 1 || std::find(seen.begin(), seen.end(), dt) != seen.end()) continue;
    seen.push_back(dt);
    b += r(rows * dt * ((nint_pad + dt - 1) / dt), sizeof(float2));  // resampled sums: FP32
  }
  b += r(p->dt.size(), 8) + r(p->dt.size(), 4);
  const int64_t img_cap = std::max<int64_t>(count_images(p, p->max_nint), 1);
  b += r(img_cap, sizeof(int4)) + r(img_cap, sizeof(Group)) + r(img_cap, 8) + r(img_cap, sizeof(DevCand)) + 4 + 4;  // candidate count, error flag
  const size_t per_slot = (size_t)p->ncol * N * sizeof(float2);
  if (slots <= 0) slots = (int)std::min<size_t>(kTBudgetBytes / per_slot, (size_t)img_cap);
  const int B = p->shape.images_per_group;
  slots = std::max(std::min(slots, 32768), B);
  const int gslots = std::max(2 * ((slots + B - 1) / B), 1);
  b += r((size_t)slots * per_slot, 1) + r((size_t)slots * p->shape.partials_per_image, sizeof(StatPartial)) +
       r((size_t)gslots * std::max(p->n_cells, 1) * 32, sizeof(float2)) + r((size_t)slots * p->ncol, 4) +
       r(slots, 4);
  if (p->flags & RF_NOISE_CLIPPED) b += r(slots, sizeof(float2));
  const int ci = rf::fused_chunk_images((int)N);
  if (ci > 0) {
    b += r(img_cap, sizeof(rf::FusedChunk)) + r(1 + 2 * gslots * ((B + ci - 1) / ci), 4);
    b += r((size_t)kDefaultRing * ci * per_slot, 1);
  }
  const size_t per_int = rows * p->npol * sizeof(float2);
  const size_t stage_nint = std::max<size_t>(1, std::min<size_t>(kStageBytes / per_int, (size_t)p->max_nint));
  b += r(stage_nint * per_int, 1);
  return b;
}

rf_status alloc_device(rf_plan* p) {
  const int N = p->npix;
  auto up = [&](auto** dst, const auto& vec) -> rf_status {
    using T = typename std::decay<decltype(vec[0])>::type;
    T* d = nullptr;
    rf_status s = p->dalloc(&d, vec.size());
    if (s != RF_OK) return s;
    if (!vec.empty()) RF_CUDA(cudaMemcpy(d, vec.data(), vec.size() * sizeof(T), cudaMemcpyHostToDevice));
    *dst = d;
    return RF_OK;
  };
  int32_t *d_delays = nullptr, *d_dt = nullptr, *d_ogc = nullptr, *d_ccp = nullptr, *d_crow = nullptr,
          *d_rptr = nullptr, *d_runs = nullptr;
  float2* d_rtw = nullptr;
  int2* d_ranges = nullptr;
  GridEntry* d_ent = nullptr;
  rf_status s;
  if ((s = up(&d_delays, p->delays)) != RF_OK) return s;
  std::vector<int32_t> dtv(p->dt.begin(), p->dt.end());
  if ((s = up(&d_dt, dtv)) != RF_OK) return s;
  if ((s = up(&d_ranges, p->ranges)) != RF_OK) return s;
  if ((s = up(&d_ccp, p->col_cell_ptr)) != RF_OK) return s;
  if ((s = up(&d_crow, p->cell_row)) != RF_OK) return s;
  if ((s = up(&d_rptr, p->col_run_ptr)) != RF_OK) return s;
  if ((s = up(&d_runs, p->col_runs)) != RF_OK) return s;
  if ((s = up(&d_rtw, p->col_run_tw)) != RF_OK) return s;
  if ((s = up(&d_ent, p->ent)) != RF_OK) return s;
  if ((s = up(&d_ogc, p->ongrid_chan)) != RF_OK) return s;
  std::vector<float2> tw(rf::fft_twiddle_len(N));
  rf::fft_twiddle_table(N, tw.data());
  float2* d_tw = nullptr;
  if ((s = up(&d_tw, tw)) != RF_OK) return s;
  float2* d_twc = d_tw;  // the column pass's sub-transform table
  if (rf::col_split(N) > 1) {
    const int L = N / rf::col_split(N);
    std::vector<float2> twc(rf::fft_twiddle_len(L));
    rf::fft_twiddle_table(L, twc.data());
    if ((s = up(&d_twc, twc)) != RF_OK) return s;
  }
  p->tb.delays = d_delays;
  p->tb.dt_list = d_dt;
  p->tb.ranges = d_ranges;
  p->tb.col_cell_ptr = d_ccp;
  p->tb.cell_row = d_crow;
  p->tb.col_run_ptr = d_rptr;
  p->tb.col_runs = d_runs;
  p->tb.col_run_tw = d_rtw;
  p->tb.ent = d_ent;
  p->tb.ongrid_chan = d_ogc;
  p->tb.twiddle = d_tw;
  p->tb.twiddle_col = d_twc;

  // Stokes-I time series S[c * nbl + b][t]
  p->nint_pad = (p->max_nint + 31) / 32 * 32;
  const size_t esz = (p->flags & RF_STORE_FP16) ? 4 : 8;
  unsigned char* dS = nullptr;
  if ((s = p->dalloc(&dS, (size_t)p->nbl * p->nchan * p->nint_pad * esz)) != RF_OK) return s;
  p->d_S = dS;
  // resampled series per dt (phase-split; FP32 sums whatever the storage of S)
  p->d_sdt.assign(p->ndt, nullptr);
  p->sdt_lp.assign(p->ndt, 0);
  std::vector<unsigned long long> sdt_addr(p->ndt, 0);
  for (int k = 0; k < p->ndt; ++k) {
    const int dt = p->dt[k];
    const int lp = (p->nint_pad + dt - 1) / dt;
    p->sdt_lp[k] = lp;
    if (dt == 1) {
      p->d_sdt[k] = dS;
    } else {
      bool same = false;
      for (int k2 = 0; k2 < k; ++k2)
        if (p->dt[k2] == dt) {
          p->d_sdt[k] = p->d_sdt[k2];
          same = true;
        }
      if (!same) {
        unsigned char* b = nullptr;
        if ((s = p->dalloc(&b, (size_t)p->nbl * p->nchan * dt * lp * sizeof(float2))) != RF_OK) return s;
        p->d_sdt[k] = b;
      }
    }
    sdt_addr[k] = (unsigned long long)(uintptr_t)p->d_sdt[k];
  }
  unsigned long long* d_sdt_addr = nullptr;
  int32_t* d_sdt_lp = nullptr;
  if ((s = up(&d_sdt_addr, sdt_addr)) != RF_OK) return s;
  if ((s = up(&d_sdt_lp, p->sdt_lp)) != RF_OK) return s;
  p->tb.sdt_ptr = d_sdt_addr;
  p->tb.sdt_lp = d_sdt_lp;

  // image lists for the largest segment
  const int64_t nimg_max = count_images(p, p->max_nint);
  if (nimg_max > (1ll << 30)) return fail(RF_ERR_INVALID_ARG, "too many images per segment (%lld)", (long long)nimg_max);
  p->img_cap = (int)std::max<int64_t>(nimg_max, 1);
  p->group_cap = p->img_cap;  // at most one group per image
  if ((s = p->dalloc(&p->d_img_info, p->img_cap)) != RF_OK) return s;
  if ((s = p->dalloc(&p->d_groups, p->group_cap)) != RF_OK) return s;
  if ((s = p->dalloc(&p->d_weight, p->img_cap)) != RF_OK) return s;
  if ((s = p->dalloc(&p->d_cands, p->img_cap)) != RF_OK) return s;
  if ((s = p->dalloc(&p->d_ncand, 1)) != RF_OK) return s;
  if ((s = p->dalloc(&p->d_err, 1)) != RF_OK) return s;
  RF_CUDA(cudaMemset(p->d_err, 0, sizeof(int)));

  // column-FFT scratch, whole groups per wave
  p->chunk_images = rf::fused_chunk_images(N);
  if (p->chunk_images > 0 && (s = p->dalloc(&p->d_chunks, (size_t)p->img_cap)) != RF_OK) return s;
  const size_t per_slot = (size_t)p->ncol * N * sizeof(float2);
  int slots = (int)std::min<size_t>(kTBudgetBytes / per_slot, (size_t)p->img_cap);
  if ((s = alloc_wave_scratch(p, slots)) != RF_OK) return s;
  if ((s = alloc_ring(p, kDefaultRing)) != RF_OK) return s;

  // host->device staging of raw visibilities
  const size_t per_int = (size_t)p->nbl * p->nchan * p->npol * sizeof(float2);
  p->stage_nint = (int)std::max<size_t>(1, std::min<size_t>(kStageBytes / per_int, (size_t)p->max_nint));
  if ((s = p->dalloc(&p->d_stage, (size_t)p->stage_nint * p->nbl * p->nchan * p->npol)) != RF_OK) return s;
  return RF_OK;
}

SegmentGeom geom(const rf_plan* p, int nint) {
  SegmentGeom g;
  g.nint = nint;
  g.nint_pad = p->nint_pad;
  g.nbl = p->nbl;
  g.nchan = p->nchan;
  g.npix = p->npix;
  g.ncol = p->ncol;
  g.ndm = p->ndm;
  g.max_cells = p->max_cells;
  g.ncells = p->n_cells;
  g.nranges = (int)p->ranges.size();
  g.partial = (p->flags & RF_EDGE_PARTIAL) != 0;
  {
    // largest series: rows of dt * ceil(nint_pad / dt) samples
    uint64_t pitch = 0;
    for (int k = 0; k < (int)p->sdt_lp.size(); ++k)
      pitch = std::max<uint64_t>(pitch, (uint64_t)p->dt[k] * p->sdt_lp[k]);
    g.idx32 = !p->wide_index && (uint64_t)p->nbl * p->nchan * pitch < (1ull << 32);
  }
  g.fp16 = (p->flags & RF_STORE_FP16) != 0;
  g.tsplit = rf::col_split(p->npix);
  return g;
}

// Ingest the segment into S.  Device input is read in place.  Page-locked
// host input that the device can address (cudaHostAlloc / cudaHostRegister
// memory, mapped into the device's address space) is also read in place by
// the ingest kernel, over the host link, with no staging copy.  Other host
// memory goes through the staging buffer in chunks.
rf_status ingest(rf_plan* p, const void* vis, int nint, cudaStream_t st) {
  cudaPointerAttributes attr;
  bool on_device = false;
  const void* mapped = nullptr;
  if (cudaPointerGetAttributes(&attr, vis) == cudaSuccess) {
    on_device = attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
    if (on_device && attr.type == cudaMemoryTypeDevice && attr.device != p->device)
      return fail(RF_ERR_INVALID_ARG, "vis is on device %d, plan is on device %d", attr.device, p->device);
    if (attr.type == cudaMemoryTypeHost && attr.devicePointer != nullptr &&
        (uintptr_t)attr.devicePointer % 16 == 0)
      mapped = attr.devicePointer;
  } else {
    cudaGetLastError();
  }
  const SegmentGeom g = geom(p, nint);
  if (on_device) {
    if ((uintptr_t)vis % 16 != 0) return fail(RF_ERR_INVALID_ARG, "device vis must be 16-byte aligned");
    RF_TIMED(p->prof, K_INGEST, st, rf::launch_ingest(static_cast<const float2*>(vis), nint, 0, p->npol, g, p->d_S, st));
  } else if (mapped) {
    RF_TIMED(p->prof, K_INGEST, st,
             rf::launch_ingest(static_cast<const float2*>(mapped), nint, 0, p->npol, g, p->d_S, st));
  } else {
    const size_t per_int = (size_t)p->nbl * p->nchan * p->npol * sizeof(float2);
    const unsigned char* src = static_cast<const unsigned char*>(vis);
    for (int t = 0; t < nint; t += p->stage_nint) {
      const int nt = std::min(p->stage_nint, nint - t);
      RF_TIMED(p->prof, K_H2D, st,
               cudaMemcpyAsync(p->d_stage, src + (size_t)t * per_int, (size_t)nt * per_int, cudaMemcpyHostToDevice,
                               st));
      RF_TIMED(p->prof, K_INGEST, st, rf::launch_ingest(p->d_stage, nt, t, p->npol, g, p->d_S, st));
    }
  }
  if (p->flags & RF_MEAN_SUBTRACT) RF_TIMED(p->prof, K_MEAN_SUBTRACT, st, rf::launch_mean_subtract(g, p->d_S, st));
  return RF_OK;
}

// Resampled series for every dt > 1 of the plan (after ingest).
rf_status resample_all(rf_plan* p, int nint, cudaStream_t st) {
  const SegmentGeom g = geom(p, nint);
  for (int k = 0; k < p->ndt; ++k) {
    if (p->dt[k] == 1 || p->d_sdt[k] == p->d_S) continue;
    bool done = false;
    for (int k2 = 0; k2 < k; ++k2) done = done || p->d_sdt[k2] == p->d_sdt[k];
    if (done) continue;
    RF_TIMED(p->prof, K_RESAMPLE, st, rf::launch_resample(g, p->d_S, p->d_sdt[k], p->dt[k], p->sdt_lp[k], st));
  }
  return RF_OK;
}

// Overlapped waves (RF_TUNE_OVERLAP).  Wave w images into half w mod 2 of
// the column-FFT scratch (and of the partials and Parseval sums), so that
// wave w + 1's gridding and column pass, on `st`, can run while wave w's row
// pass and finalize run on the plan's second stream.  Each pass does the same
// arithmetic on the same image as in the serial order and the finalizes keep
// their order, so results are identical.  The column pass takes the higher
// priority and at most one block per SM; the row pass runs short-lived blocks
// of kOverlapRowItems work items, which fill whatever the column pass leaves.
// Before a half is reused its previous wave's row pass and finalize must be
// done (an event per half); the caller's stream waits for the last finalize.
rf_status overlapped_loop(rf_plan* p, const SegmentGeom& g, const std::vector<Wave>& waves, DevStat* d_stats,
                         cudaStream_t st, const rf::PassLaunch& pc, const rf::PassLaunch& pr);

rf_status run_waves_overlapped(rf_plan* p, const SegmentGeom& g, const std::vector<Wave>& waves,
                               DevStat* d_stats, cudaStream_t st) {
  int prio_lo = 0, prio_hi = 0;
  RF_CUDA(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
  if (!p->ostream) RF_CUDA(cudaStreamCreateWithPriority(&p->ostream, cudaStreamNonBlocking, prio_lo));
  for (cudaEvent_t& e : p->oev)
    if (!e) RF_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaStream_t so = p->ostream;
  rf::PassLaunch pc, pr;
  pc.one_per_sm = true;
  pc.set_priority = pr.set_priority = true;
  pc.priority = prio_hi;
  pr.priority = prio_lo;
  pr.items_per_block = kOverlapRowItems;
  // the caller's stream waits for the second stream however the loop ends
  // (a failed launch leaves no work of the plan unjoined behind the call)
  const rf_status s = overlapped_loop(p, g, waves, d_stats, st, pc, pr);
  const bool joined =
      cudaEventRecord(p->oev[4], so) == cudaSuccess && cudaStreamWaitEvent(st, p->oev[4], 0) == cudaSuccess;
  if (s != RF_OK) return s;
  if (!joined)
    return fail(RF_ERR_CUDA, "joining the overlapped waves' streams: %s", cudaGetErrorString(cudaGetLastError()));
  return RF_OK;
}

// The wave loop of run_waves_overlapped (streams and events set up).
rf_status overlapped_loop(rf_plan* p, const SegmentGeom& g, const std::vector<Wave>& waves, DevStat* d_stats,
                         cudaStream_t st, const rf::PassLaunch& pc, const rf::PassLaunch& pr) {
  cudaStream_t so = p->ostream;
  const size_t half = (size_t)p->slots_max / 2;
  const size_t per_slot = (size_t)p->ncol * p->npix;
  const size_t nrb = (size_t)p->shape.partials_per_image;
  for (size_t wi = 0; wi < waves.size(); ++wi) {
    const Wave& w = waves[wi];
    const int h = (int)(wi & 1);
    const int ng = w.g_end - w.g_begin;
    const int ni = w.img_end - w.img_begin;
    float2* T = p->d_T + h * half * per_slot;
    StatPartial* part = p->d_partials + h * half * nrb;
    float* colsq = p->d_colsq + h * half * p->ncol;
    float* mean0 = p->d_mean0 + h * half;
    RF_TIMED(p->prof, K_GRID_CELLS, st,
             rf::launch_grid_cells(g, p->tb, p->d_groups, w.g_begin, ng, p->d_cellbuf, st));
    if (wi >= 2) RF_CUDA(cudaStreamWaitEvent(st, p->oev[2 + h], 0));
    RF_TIMED(p->prof, K_GRID_COLFFT, st,
             rf::launch_colfft(g, p->tb, p->d_groups, w.g_begin, ng, w.img_begin, p->d_cellbuf, T, colsq, mean0,
                               st, &pc));
    RF_CUDA(cudaEventRecord(p->oev[h], st));
    RF_CUDA(cudaStreamWaitEvent(so, p->oev[h], 0));
    RF_TIMED(p->prof, K_ROWFFT_STATS, so,
             rf::launch_rowfft_stats(g, p->tb, T, ni, w.img_begin, p->d_weight, part, nullptr,
                                     p->tmap_H[h].nbox > 0 ? &p->tmap_H[h] : nullptr, p->d_err, so, nullptr,
                                     &pr));
    RF_TIMED(p->prof, K_FINALIZE, so,
             rf::launch_finalize(g, part, colsq, mean0, p->d_img_info, p->d_weight, ni, w.img_begin, p->threshold,
                                 p->d_cands, p->d_ncand, p->img_cap, d_stats, so, false));
    RF_CUDA(cudaEventRecord(p->oev[2 + h], so));
  }
  return RF_OK;
}

// Pass A / pass B / finalize over the image list currently on the device.
rf_status run_waves(rf_plan* p, int nint, const std::vector<Wave>& waves, int nimg_total, DevStat* d_stats,
                    float* d_images, cudaStream_t st) {
  const SegmentGeom g = geom(p, nint);
  RF_TIMED(p->prof, K_WEIGHTS, st,
           rf::launch_weights(p->d_img_info, nimg_total, (p->flags & RF_EDGE_PARTIAL) != 0, g, p->tb,
                              (double)p->n_on, p->d_weight, st));
  const bool fused = d_images == nullptr && &waves == &p->waves && use_fused(p);
  if (!fused && d_images == nullptr && &waves == &p->waves && p->waves_overlap && overlap_possible(p))
    return run_waves_overlapped(p, g, waves, d_stats, st);
  for (size_t wi = 0; wi < waves.size(); ++wi) {
    const Wave& w = waves[wi];
    const int ng = w.g_end - w.g_begin;
    const int ni = w.img_end - w.img_begin;
    RF_TIMED(p->prof, K_GRID_CELLS, st,
             rf::launch_grid_cells(g, p->tb, p->d_groups, w.g_begin, ng, p->d_cellbuf, st));
    if (fused) {
      const int2 wc = p->wave_chunks[wi];
      RF_TIMED(p->prof, K_IMAGE_FUSED, st,
               rf::launch_image_fused(g, p->tb, p->d_groups, w.g_begin, p->d_chunks + wc.x, wc.y - wc.x,
                                      w.img_begin, p->d_cellbuf, p->d_Tring, p->ring, p->tmap_ring, p->d_colsq,
                                      p->d_mean0, p->d_partials, p->d_fcount, p->d_err, st));
      RF_TIMED(p->prof, K_FINALIZE, st,
               rf::launch_finalize(g, p->d_partials, p->d_colsq, p->d_mean0, p->d_img_info, p->d_weight, ni,
                                   w.img_begin, p->threshold, p->d_cands, p->d_ncand, p->img_cap, d_stats, st,
                                   false));
      continue;
    }
    RF_TIMED(p->prof, K_GRID_COLFFT, st,
             rf::launch_colfft(g, p->tb, p->d_groups, w.g_begin, ng, w.img_begin, p->d_cellbuf, p->d_T,
                               p->d_colsq, p->d_mean0, st));
    const bool clip = (p->flags & RF_NOISE_CLIPPED) != 0;
    if (clip)
      RF_TIMED(p->prof, K_CLIP_WINDOW, st, rf::launch_clip_window(g, p->d_colsq, p->d_mean0, ni, p->d_clip, st));
    float* im = d_images ? d_images + (size_t)w.img_begin * p->npix * p->npix : nullptr;
    RF_TIMED(p->prof, K_ROWFFT_STATS, st,
             rf::launch_rowfft_stats(g, p->tb, p->d_T, ni, w.img_begin, p->d_weight, p->d_partials, im,
                                     p->tmap_T.nbox > 0 ? &p->tmap_T : nullptr, p->d_err, st,
                                     clip ? p->d_clip : nullptr));
    RF_TIMED(p->prof, K_FINALIZE, st,
             rf::launch_finalize(g, p->d_partials, p->d_colsq, p->d_mean0, p->d_img_info, p->d_weight, ni,
                                 w.img_begin, p->threshold, p->d_cands, p->d_ncand, p->img_cap, d_stats, st,
                                 clip));
  }
  return RF_OK;
}

// The batched wave loop through a CUDA graph: captured on the plan's
// private stream the first time an image list is searched (per nint and
// stats output) and replayed afterwards.  With profiling on, searches use
// direct launches instead (events in a graph do not time its kernels).  The private
// stream is ordered after the caller's stream and the caller's stream after
// the replay, so the call behaves like direct launches on `st`.
rf_status run_waves_graph(rf_plan* p, int nint, int nimg, DevStat* d_stats, cudaStream_t st) {
  if (!p->gstream) {
    RF_CUDA(cudaStreamCreateWithFlags(&p->gstream, cudaStreamNonBlocking));
    RF_CUDA(cudaEventCreateWithFlags(&p->join[0], cudaEventDisableTiming));
    RF_CUDA(cudaEventCreateWithFlags(&p->join[1], cudaEventDisableTiming));
  }
  auto& gc = p->graph;
  const bool want_stats = d_stats != nullptr;
  if (!(gc.valid && gc.nint == nint && gc.stats == want_stats && gc.prof == p->prof.on)) {
    p->drop_graph();
    const size_t u0 = p->prof.used;
    RF_CUDA(cudaStreamBeginCapture(p->gstream, cudaStreamCaptureModeThreadLocal));
    rf_status s = run_waves(p, nint, p->waves, nimg, d_stats, nullptr, p->gstream);
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(p->gstream, &g);
    if (s != RF_OK) {
      if (g) cudaGraphDestroy(g);
      p->prof.take(u0, &gc.ev, &gc.kind);
      p->drop_graph();
      return s;
    }
    if (ec != cudaSuccess) return fail(RF_ERR_CUDA, "graph capture: %s", cudaGetErrorString(ec));
    // overlapped waves carry per-launch priorities on their kernel nodes
    const cudaError_t ei =
        cudaGraphInstantiate(&gc.exec, g, p->waves_overlap ? cudaGraphInstantiateFlagUseNodePriority : 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return fail(RF_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(ei));
    p->prof.take(u0, &gc.ev, &gc.kind);
    gc.valid = true;
    gc.nint = nint;
    gc.stats = want_stats;
    gc.prof = p->prof.on;
  }
  RF_CUDA(cudaEventRecord(p->join[0], st));
  RF_CUDA(cudaStreamWaitEvent(p->gstream, p->join[0], 0));
  RF_CUDA(cudaGraphLaunch(gc.exec, p->gstream));
  RF_CUDA(cudaEventRecord(p->join[1], p->gstream));
  RF_CUDA(cudaStreamWaitEvent(st, p->join[1], 0));
  p->graph_pending = gc.prof;
  return RF_OK;
}

// Plain form buffers, sized for chunks of up to `cap` images within the budget.
rf_status alloc_plain(rf_plan* p) {
  if (p->plain.cap > 0) return RF_OK;
  const size_t N = p->npix;
  const size_t per = (size_t)p->nbl * p->nchan * sizeof(float2) + N * (N / 2 + 1) * sizeof(float2) +
                     (N / 2) * N * sizeof(float2) + N * N * sizeof(float) +
                     (size_t)p->shape.partials_per_image * sizeof(StatPartial);
  const int cap = (int)std::max<size_t>(1, std::min<size_t>(kPlainBudgetBytes / per, 4096));
  rf_status s;
  rf::PlainBuffers& b = p->plain;
  if ((s = p->dalloc(&b.R, (size_t)p->nbl * p->nchan * cap)) != RF_OK) return s;
  if ((s = p->dalloc(&b.grid, (size_t)cap * N * (N / 2 + 1))) != RF_OK) return s;
  if ((s = p->dalloc(&b.T, (size_t)cap * (N / 2) * N)) != RF_OK) return s;
  if ((s = p->dalloc(&b.images, (size_t)cap * N * N)) != RF_OK) return s;
  if ((s = p->dalloc(&b.partials, (size_t)cap * p->shape.partials_per_image)) != RF_OK) return s;
  int4* d_ent = nullptr;
  if ((s = p->dalloc(&d_ent, p->plain_ent.size())) != RF_OK) return s;
  if (!p->plain_ent.empty())
    RF_CUDA(cudaMemcpy(d_ent, p->plain_ent.data(), p->plain_ent.size() * sizeof(int4), cudaMemcpyHostToDevice));
  b.S = p->d_S;
  b.ent = d_ent;
  b.nent = (int)p->plain_ent.size();
  b.cap = cap;
  return RF_OK;
}

// The plain form: for each (DM, dt) trial, chunks of its images through the
// unfused launch set.
rf_status run_plain(rf_plan* p, int nint, DevStat* d_stats, cudaStream_t st) {
  rf_status s = alloc_plain(p);
  if (s != RF_OK) return s;
  const SegmentGeom g = geom(p, nint);
  const int nimg_total = (int)p->img_info.size();
  RF_TIMED(p->prof, K_WEIGHTS, st,
           rf::launch_weights(p->d_img_info, nimg_total, (p->flags & RF_EDGE_PARTIAL) != 0, g, p->tb,
                              (double)p->n_on, p->d_weight, st));
  int img0 = 0;
  for (int d = 0; d < p->ndm; ++d)
    for (int sdt = 0; sdt < p->ndt; ++sdt) {
      const int nt = n_times(p, nint, d, sdt);
      for (int t0 = 0; t0 < nt; t0 += p->plain.cap) {
        const int nk = std::min(p->plain.cap, nt - t0);
        RF_TIMED(p->prof, K_PLAIN_TRIAL, st,
                 rf::launch_plain_chunk(g, p->tb, p->plain, d, sdt, t0, nk, img0, p->d_img_info, p->d_weight,
                                        p->threshold, p->d_cands, p->d_ncand, p->img_cap, d_stats, st,
                                        (p->flags & RF_NOISE_CLIPPED) != 0));
        img0 += nk;
      }
    }
  return RF_OK;
}

// Sets the plan's t' span for one search and clears it on every exit.
struct SpanGuard {
  rf_plan* p;
  SpanGuard(rf_plan* pl, int span) : p(pl) { p->t_span = span; }
  ~SpanGuard() { p->t_span = 0; }
};

rf_status search_impl(rf_plan* p, const void* vis, int nint, void* stream, rf_candidate* out, size_t cap,
                      size_t* n_out, bool want_stats, rf_image_stat* stats, size_t stats_cap, size_t* n_stats,
                      int span = 0) {
  if (!p) return fail(RF_ERR_INVALID_ARG, "plan is NULL");
  if (p->host_only) return fail(RF_ERR_INVALID_ARG, "plan was created with RF_HOST_ONLY");
  if (!vis) return fail(RF_ERR_INVALID_ARG, "vis is NULL");
  if (!n_out) return fail(RF_ERR_INVALID_ARG, "n_out is NULL");
  if (cap > 0 && !out) return fail(RF_ERR_INVALID_ARG, "out is NULL with cap > 0");
  if (nint < 1 || nint > p->max_nint) return fail(RF_ERR_SHAPE, "nint %d out of [1, %d]", nint, p->max_nint);
  BusyGuard bg(&p->busy);
  if (!bg.owned) return fail(RF_ERR_BUSY, "plan is in use by another call");
  DeviceGuard dg(p->device);
  if (!dg.ok) return fail(RF_ERR_CUDA, "cannot select device %d", p->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  *n_out = 0;
  SpanGuard sg(p, span);

  rf_status s = ingest(p, vis, nint, st);
  if (s != RF_OK) return s;
  s = resample_all(p, nint, st);
  if (s != RF_OK) return s;
  if (p->cached_nint != nint || p->cached_span != p->t_span) {
    build_lists(p, nint);
    if (!p->img_info.empty()) {
      RF_CUDA(cudaMemcpyAsync(p->d_img_info, p->img_info.data(), p->img_info.size() * sizeof(int4),
                              cudaMemcpyHostToDevice, st));
      RF_CUDA(cudaMemcpyAsync(p->d_groups, p->groups.data(), p->groups.size() * sizeof(Group),
                              cudaMemcpyHostToDevice, st));
      if (!p->chunks.empty())
        RF_CUDA(cudaMemcpyAsync(p->d_chunks, p->chunks.data(), p->chunks.size() * sizeof(rf::FusedChunk),
                                cudaMemcpyHostToDevice, st));
    }
  }
  const int nimg = (int)p->img_info.size();
  DevStat* d_stats = nullptr;
  if (want_stats && stats) {
    if (!p->d_stats) {
      s = p->dalloc(&p->d_stats, p->img_cap);
      if (s != RF_OK) return s;
    }
    d_stats = p->d_stats;
  }
  RF_CUDA(cudaMemsetAsync(p->d_ncand, 0, sizeof(int), st));
  if (nimg > 0) {
    if (p->form == RF_FORM_PLAIN)
      s = run_plain(p, nint, d_stats, st);
    else if (p->use_graphs && !p->prof.on)  // per-kernel event timing needs direct launches
      s = run_waves_graph(p, nint, nimg, d_stats, st);
    else
      s = run_waves(p, nint, p->waves, nimg, d_stats, nullptr, st);
    if (s != RF_OK) return s;
  }
  int ncand = 0, kerr = 0;
  RF_CUDA(cudaMemcpyAsync(&ncand, p->d_ncand, sizeof(int), cudaMemcpyDeviceToHost, st));
  RF_CUDA(cudaMemcpyAsync(&kerr, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  RF_CUDA(cudaStreamSynchronize(st));
  if (kerr) {
    cudaMemset(p->d_err, 0, sizeof(int));
    return fail(RF_ERR_TIMEOUT, "a bounded device-side wait (a tile copy, or a fused-pass dependency) gave up");
  }
  ncand = std::min(ncand, p->img_cap);
  std::vector<DevCand> dc(ncand);
  if (ncand > 0)
    RF_CUDA(cudaMemcpyAsync(dc.data(), p->d_cands, ncand * sizeof(DevCand), cudaMemcpyDeviceToHost, st));
  std::vector<DevStat> ds;
  if (d_stats && nimg > 0) {
    ds.resize(nimg);
    RF_CUDA(cudaMemcpyAsync(ds.data(), d_stats, (size_t)nimg * sizeof(DevStat), cudaMemcpyDeviceToHost, st));
  }
  RF_CUDA(cudaStreamSynchronize(st));
  p->prof.collect();
  if (p->graph_pending) {
    p->prof.add_pairs(p->graph.ev, p->graph.kind);
    p->graph_pending = false;
  }
  std::sort(dc.begin(), dc.end(), [](const DevCand& a, const DevCand& b) {
    if (a.d != b.d) return a.d < b.d;
    if (a.s != b.s) return a.s < b.s;
    return a.t < b.t;
  });
  const int half = p->npix / 2;
  const size_t nw = std::min<size_t>(cap, dc.size());
  for (size_t k = 0; k < nw; ++k) {
    rf_candidate& c = out[k];
    c.dm_idx = dc[k].d;
    c.dt_idx = dc[k].s;
    c.t_idx = dc[k].t;
    c.x = dc[k].x;
    c.y = dc[k].y;
    c.snr = dc[k].snr;
    c.peak = dc[k].peak;
    c.sigma = dc[k].sigma;
    c.dm = p->dm[dc[k].d];
    c.l_rad = (double)(dc[k].x - half) * p->cell;
    c.m_rad = (double)(dc[k].y - half) * p->cell;
  }
  *n_out = dc.size();
  if (want_stats && n_stats) *n_stats = (size_t)nimg;
  if (d_stats) {
    const size_t ns = std::min<size_t>(stats_cap, (size_t)nimg);
    for (size_t k = 0; k < ns; ++k) {
      rf_image_stat& o = stats[k];
      o.dm_idx = p->img_info[k].x;
      o.dt_idx = p->img_info[k].y;
      o.t_idx = p->img_info[k].z;
      o.x = ds[k].x;
      o.y = ds[k].y;
      o.peak = ds[k].peak;
      o.sigma = ds[k].sigma;
      o.snr = ds[k].snr;
      o.mean = ds[k].mean;
      o.weight = ds[k].weight;
    }
    if ((size_t)nimg > stats_cap) return fail(RF_ERR_CAPACITY, "%d image stats, capacity %zu", nimg, stats_cap);
  }
  if (dc.size() > cap) return fail(RF_ERR_CAPACITY, "%zu candidates, capacity %zu", dc.size(), cap);
  return RF_OK;
}

// Every trial (d, s, t') must be one the plan searches at this nint.
rf_status check_trials(const rf_plan* p, int nint, const int32_t* trials, int n) {
  for (int k = 0; k < n; ++k) {
    const int d = trials[3 * k], s = trials[3 * k + 1], t = trials[3 * k + 2];
    if (d < 0 || d >= p->ndm || s < 0 || s >= p->ndt || t < 0 || t >= n_times(p, nint, d, s))
      return fail(RF_ERR_INVALID_ARG, "trial %d (%d, %d, %d) is not searched", k, d, s, t);
  }
  return RF_OK;
}

// Images of n trials into d_img ([n][N][N]), after ingest and resampling.
// The trials replace the plan's cached search lists.
rf_status render_core(rf_plan* p, int nint, const int32_t* trials, int n, float* d_img, cudaStream_t st) {
  if (n > p->img_cap) return fail(RF_ERR_INVALID_ARG, "at most %d images per call", p->img_cap);
  std::vector<int4> info(n);
  std::vector<Group> grp(n);
  for (int k = 0; k < n; ++k) {
    info[k] = make_int4(trials[3 * k], trials[3 * k + 1], trials[3 * k + 2], 0);
    grp[k] = Group{trials[3 * k], trials[3 * k + 1], trials[3 * k + 2], 1, k, {0, 0, 0}};
  }
  p->cached_nint = -1;
  p->drop_graph();
  RF_CUDA(cudaMemcpyAsync(p->d_img_info, info.data(), n * sizeof(int4), cudaMemcpyHostToDevice, st));
  RF_CUDA(cudaMemcpyAsync(p->d_groups, grp.data(), n * sizeof(Group), cudaMemcpyHostToDevice, st));
  std::vector<Wave> waves;
  const int per_wave = std::min(p->slots_max, p->gslots_max);  // single-image groups
  for (int k = 0; k < n; k += per_wave) {
    const int e = std::min(n, k + per_wave);
    waves.push_back(Wave{k, e, k, e});
  }
  RF_CUDA(cudaMemsetAsync(p->d_ncand, 0, sizeof(int), st));
  rf_status s = run_waves(p, nint, waves, n, nullptr, d_img, st);
  // the host-side lists above must outlive the copies
  cudaError_t e = cudaStreamSynchronize(st);
  if (s == RF_OK && e != cudaSuccess) s = fail(RF_ERR_CUDA, "render: %s", cudaGetErrorString(e));
  int kerr = 0;
  if (s == RF_OK && cudaMemcpy(&kerr, p->d_err, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess && kerr) {
    cudaMemset(p->d_err, 0, sizeof(int));
    s = fail(RF_ERR_TIMEOUT, "a row-pass tile copy did not complete within its wait limit");
  }
  return s;
}

// Device allocations freed when the scope ends (calls outside the hot path).
struct DeviceScratch {
  std::vector<void*> ptrs;
  template <typename T>
  rf_status get(T** q, size_t count) {
    void* v = nullptr;
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&v, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(RF_ERR_NO_MEMORY, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    ptrs.push_back(v);
    *q = static_cast<T*>(v);
    return RF_OK;
  }
  ~DeviceScratch() {
    for (void* v : ptrs) cudaFree(v);
  }
};

}  // namespace

namespace rf {
void set_last_error(const char* msg) { g_err = msg ? msg : ""; }

rf_status plan_geometry(const rf_plan* p, PlanGeometry* g) {
  if (!p || !g) return fail(RF_ERR_INVALID_ARG, "NULL argument");
  g->nbl = p->nbl;
  g->nchan = p->nchan;
  g->npol = p->npol;
  g->max_nint = p->max_nint;
  g->max_delay = 0;
  for (int d = 0; d < p->ndm; ++d) g->max_delay = std::max(g->max_delay, p->max_delay[d]);
  g->device = p->device;
  g->host_only = p->host_only;
  g->dt.assign(p->dt.begin(), p->dt.end());
  return RF_OK;
}

rf_status search_span(rf_plan* p, const void* vis, int nint, int span, void* stream,
                      std::vector<rf_candidate>* cands, std::vector<rf_image_stat>* stats) {
  if (!p || !cands) return fail(RF_ERR_INVALID_ARG, "NULL argument");
  if (span < 0) return fail(RF_ERR_INVALID_ARG, "span %d < 0", span);
  int64_t nimg = 0;  // images of this (nint, span): at most one candidate each
  for (int d = 0; d < p->ndm; ++d)
    for (int k = 0; k < p->ndt; ++k) nimg += n_times_span(p, nint, d, k, span);
  cands->resize((size_t)std::max<int64_t>(nimg, 1));
  size_t n_out = 0, n_stats = 0;
  rf_status s;
  if (stats) {
    stats->resize((size_t)std::max<int64_t>(nimg, 1));
    s = search_impl(p, vis, nint, stream, cands->data(), cands->size(), &n_out, true, stats->data(), stats->size(),
                    &n_stats, span);
    stats->resize(s == RF_OK ? n_stats : 0);
  } else {
    s = search_impl(p, vis, nint, stream, cands->data(), cands->size(), &n_out, false, nullptr, 0, nullptr, span);
  }
  cands->resize(s == RF_OK ? n_out : 0);
  return s;
}
}  // namespace rf

extern "C" {

const char* rf_last_error(void) { return g_err.c_str(); }

const char* rf_version(void) { return "realfast_gb300 0.1.0 (sm_103a)"; }

rf_status rf_plan_create(const rf_plan_desc* desc, rf_plan** out) {
  if (!out) return fail(RF_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  rf_status s = validate(desc);
  if (s != RF_OK) return s;
  rf_plan* p = new (std::nothrow) rf_plan();
  if (!p) return fail(RF_ERR_NO_MEMORY, "host allocation failed");
  p->nant = desc->nant;
  p->nchan = desc->nchan;
  p->npol = desc->npol;
  p->npix = desc->npix;
  p->ndm = desc->ndm;
  p->ndt = desc->ndt;
  p->max_nint = desc->max_nint;
  p->device = desc->device;
  p->flags = desc->flags;
  p->inttime = desc->inttime_s;
  p->cell = desc->cell_rad;
  p->threshold = desc->threshold_sigma;
  p->ant_uvw.assign(desc->ant_uvw_m, desc->ant_uvw_m + 3 * desc->nant);
  p->freq.assign(desc->freq_hz, desc->freq_hz + desc->nchan);
  p->dm.assign(desc->dm_list, desc->dm_list + desc->ndm);
  p->dt.assign(desc->dt_list, desc->dt_list + desc->ndt);
  p->host_only = (desc->flags & RF_HOST_ONLY) != 0;
  s = build_tables(p);
  if (s != RF_OK) {
    delete p;
    return s;
  }
  if (!p->host_only) {
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
      cudaGetLastError();
      delete p;
      return fail(RF_ERR_NO_DEVICE, "no CUDA device available");
    }
    if (p->device < 0 || p->device >= ndev) {
      delete p;
      return fail(RF_ERR_INVALID_ARG, "device %d out of [0, %d)", desc->device, ndev);
    }
    DeviceGuard dg(p->device);
    if (!dg.ok) {
      delete p;
      return fail(RF_ERR_CUDA, "cannot select device %d", desc->device);
    }
    s = alloc_device(p);
    if (s != RF_OK) {
      std::string keep = g_err;
      delete p;
      g_err = keep;
      return s;
    }
  }
  *out = p;
  return RF_OK;
}

rf_status rf_plan_estimate_bytes(const rf_plan_desc* desc, int64_t wave_images, uint64_t* bytes) {
  if (!bytes) return fail(RF_ERR_INVALID_ARG, "bytes is NULL");
  rf_status s = validate(desc);
  if (s != RF_OK) return s;
  rf_plan tmp;
  tmp.nant = desc->nant;
  tmp.nchan = desc->nchan;
  tmp.npol = desc->npol;
  tmp.npix = desc->npix;
  tmp.ndm = desc->ndm;
  tmp.ndt = desc->ndt;
  tmp.max_nint = desc->max_nint;
  tmp.flags = desc->flags;
  tmp.inttime = desc->inttime_s;
  tmp.cell = desc->cell_rad;
  tmp.ant_uvw.assign(desc->ant_uvw_m, desc->ant_uvw_m + 3 * desc->nant);
  tmp.freq.assign(desc->freq_hz, desc->freq_hz + desc->nchan);
  tmp.dm.assign(desc->dm_list, desc->dm_list + desc->ndm);
  tmp.dt.assign(desc->dt_list, desc->dt_list + desc->ndt);
  s = build_tables(&tmp);
  if (s != RF_OK) return s;
  *bytes = estimate_device_bytes(&tmp, (int)std::min<int64_t>(std::max<int64_t>(wave_images, 0), 32768));
  return RF_OK;
}

rf_status rf_plan_destroy(rf_plan* plan) {
  if (!plan) return RF_OK;
  if (plan->busy.load() != 0) return fail(RF_ERR_BUSY, "plan is in use");
  delete plan;
  return RF_OK;
}

rf_status rf_search_segment(rf_plan* plan, const void* vis, int32_t nint, void* stream, rf_candidate* out,
                            size_t cap, size_t* n_out) {
  return search_impl(plan, vis, nint, stream, out, cap, n_out, false, nullptr, 0, nullptr);
}

rf_status rf_search_segment_stats(rf_plan* plan, const void* vis, int32_t nint, void* stream, rf_candidate* out,
                                  size_t cap, size_t* n_out, rf_image_stat* stats, size_t stats_cap,
                                  size_t* n_stats) {
  if (!stats && stats_cap > 0) return fail(RF_ERR_INVALID_ARG, "stats is NULL with stats_cap > 0");
  return search_impl(plan, vis, nint, stream, out, cap, n_out, true, stats, stats_cap, n_stats);
}

rf_status rf_render_images(rf_plan* p, const void* vis, int32_t nint, void* stream, const int32_t* trials,
                           int32_t n, float* images) {
  if (!p) return fail(RF_ERR_INVALID_ARG, "plan is NULL");
  if (p->host_only) return fail(RF_ERR_INVALID_ARG, "plan was created with RF_HOST_ONLY");
  if (!vis || !trials || !images || n < 1) return fail(RF_ERR_INVALID_ARG, "bad render arguments");
  if (nint < 1 || nint > p->max_nint) return fail(RF_ERR_SHAPE, "nint %d out of [1, %d]", nint, p->max_nint);
  if (n > p->img_cap) return fail(RF_ERR_INVALID_ARG, "at most %d images per call", p->img_cap);
  rf_status s = check_trials(p, nint, trials, n);
  if (s != RF_OK) return s;
  BusyGuard bg(&p->busy);
  if (!bg.owned) return fail(RF_ERR_BUSY, "plan is in use by another call");
  DeviceGuard dg(p->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s = ingest(p, vis, nint, st);
  if (s != RF_OK) return s;
  s = resample_all(p, nint, st);
  if (s != RF_OK) return s;
  const size_t npx = (size_t)p->npix * p->npix;
  float* d_img = nullptr;
  cudaError_t e = cudaMalloc(&d_img, (size_t)n * npx * sizeof(float));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(RF_ERR_NO_MEMORY, "render buffer: %s", cudaGetErrorString(e));
  }
  s = render_core(p, nint, trials, n, d_img, st);
  if (s == RF_OK) {
    e = cudaMemcpyAsync(images, d_img, (size_t)n * npx * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = fail(RF_ERR_CUDA, "render copy: %s", cudaGetErrorString(e));
  }
  cudaStreamSynchronize(st);
  p->prof.collect();
  cudaFree(d_img);
  return s;
}

rf_status rf_candidate_products(rf_plan* p, const void* vis, int32_t nint, void* stream, const rf_candidate* cands,
                                int32_t n, rf_candidate_features* features, float* spectra, float* images) {
  if (!p) return fail(RF_ERR_INVALID_ARG, "plan is NULL");
  if (p->host_only) return fail(RF_ERR_INVALID_ARG, "plan was created with RF_HOST_ONLY");
  if (!vis || !cands || !features || n < 1) return fail(RF_ERR_INVALID_ARG, "bad candidate-product arguments");
  if (nint < 1 || nint > p->max_nint) return fail(RF_ERR_SHAPE, "nint %d out of [1, %d]", nint, p->max_nint);
  std::vector<int32_t> trials(3 * (size_t)n);
  std::vector<rf::CandRef> refs(n);
  for (int k = 0; k < n; ++k) {
    const rf_candidate& c = cands[k];
    if (c.x < 0 || c.x >= p->npix || c.y < 0 || c.y >= p->npix)
      return fail(RF_ERR_INVALID_ARG, "candidate %d pixel (%d, %d) outside the image", k, c.x, c.y);
    trials[3 * k] = c.dm_idx;
    trials[3 * k + 1] = c.dt_idx;
    trials[3 * k + 2] = c.t_idx;
    refs[k] = rf::CandRef{c.dm_idx, c.dt_idx, c.t_idx, c.x, c.y, {0, 0, 0}};
  }
  rf_status s = check_trials(p, nint, trials.data(), n);
  if (s != RF_OK) return s;
  BusyGuard bg(&p->busy);
  if (!bg.owned) return fail(RF_ERR_BUSY, "plan is in use by another call");
  DeviceGuard dg(p->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  s = ingest(p, vis, nint, st);
  if (s != RF_OK) return s;
  s = resample_all(p, nint, st);
  if (s != RF_OK) return s;
  if (!p->d_cellbc) {  // per-row (iu, iv) table, built on first use
    std::vector<int2> cb((size_t)p->nbl * p->nchan);
    for (int b = 0; b < p->nbl; ++b)
      for (int c = 0; c < p->nchan; ++c) {
        const size_t k = (size_t)b * p->nchan + c;
        cb[(size_t)c * p->nbl + b] = p->ongrid[k] ? make_int2(p->iu[k], p->iv[k]) : make_int2(rf::kOffGrid, 0);
      }
    s = p->dalloc(&p->d_cellbc, cb.size());
    if (s != RF_OK) return s;
    RF_CUDA(cudaMemcpyAsync(p->d_cellbc, cb.data(), cb.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
  }
  const size_t npx = (size_t)p->npix * p->npix;
  const size_t nch = (size_t)p->nchan;
  // scratch: refs, FP64 spectra and weights, FP32 spectra, moments; images in chunks
  const int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)n, (size_t)(1ull << 30) / (npx * sizeof(float))));
  DeviceScratch sc;
  rf::CandRef* d_refs = nullptr;
  double2* d_spec = nullptr;
  double* d_wch = nullptr;
  float2* d_spec32 = nullptr;
  double* d_smom = nullptr;
  double* d_imom = nullptr;
  double* d_mpart = nullptr;
  float* d_img = nullptr;
  if ((s = sc.get(&d_refs, n)) != RF_OK || (s = sc.get(&d_spec, n * nch)) != RF_OK ||
      (s = sc.get(&d_wch, n * nch)) != RF_OK || (s = sc.get(&d_smom, (size_t)n * 6)) != RF_OK ||
      (s = sc.get(&d_imom, (size_t)n * 4)) != RF_OK || (s = sc.get(&d_img, (size_t)chunk * npx)) != RF_OK)
    return s;
  const int mslices = rf::image_moment_slices(chunk, npx);
  if ((s = sc.get(&d_mpart, (size_t)chunk * mslices * 4)) != RF_OK) return s;
  if (spectra && (s = sc.get(&d_spec32, n * nch)) != RF_OK) return s;
  RF_CUDA(cudaMemcpyAsync(d_refs, refs.data(), n * sizeof(rf::CandRef), cudaMemcpyHostToDevice, st));
  const SegmentGeom g = geom(p, nint);
  RF_CUDA(rf::launch_cand_spectrum(g, p->tb, p->d_cellbc, d_refs, n, d_spec, d_wch, d_spec32, d_smom, st));
  for (int k0 = 0; k0 < n; k0 += chunk) {
    const int m = std::min(chunk, n - k0);
    s = render_core(p, nint, trials.data() + 3 * (size_t)k0, m, d_img, st);
    if (s != RF_OK) return s;
    RF_CUDA(rf::launch_image_moments(d_img, m, npx, mslices, d_mpart, d_imom + (size_t)k0 * 4, st));
    if (images)
      RF_CUDA(cudaMemcpyAsync(images + (size_t)k0 * npx, d_img, (size_t)m * npx * sizeof(float),
                              cudaMemcpyDeviceToHost, st));
  }
  std::vector<double> smom((size_t)n * 6), imom((size_t)n * 4);
  RF_CUDA(cudaMemcpyAsync(smom.data(), d_smom, smom.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  RF_CUDA(cudaMemcpyAsync(imom.data(), d_imom, imom.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (spectra)
    RF_CUDA(cudaMemcpyAsync(spectra, d_spec32, n * nch * sizeof(float2), cudaMemcpyDeviceToHost, st));
  RF_CUDA(cudaStreamSynchronize(st));
  p->prof.collect();
  for (int k = 0; k < n; ++k) {
    rf_candidate_features& f = features[k];
    f.dm_idx = refs[k].d;
    f.dt_idx = refs[k].s;
    f.t_idx = refs[k].t;
    f.x = refs[k].x;
    f.y = refs[k].y;
    f.nchan_used = (int32_t)smom[6 * k + 5];
    f.image_mean = imom[4 * k];
    f.image_sigma = imom[4 * k + 1];
    f.image_skew = imom[4 * k + 2];
    f.image_kurtosis = imom[4 * k + 3];
    f.spec_mean = smom[6 * k];
    f.spec_std = smom[6 * k + 1];
    f.spec_skew = smom[6 * k + 2];
    f.spec_kurtosis = smom[6 * k + 3];
    f.peak_from_spectrum = smom[6 * k + 4];
  }
  return RF_OK;
}

rf_status rf_periodicity_search(rf_plan* p, const void* vis, int32_t nint, int32_t L, int32_t kmin, int32_t kmax,
                                double threshold, void* stream, rf_periodic_candidate* out, size_t cap,
                                size_t* n_out, rf_periodic_candidate* stats, size_t stats_cap, size_t* n_stats) {
  if (!p) return fail(RF_ERR_INVALID_ARG, "plan is NULL");
  if (p->host_only) return fail(RF_ERR_INVALID_ARG, "plan was created with RF_HOST_ONLY");
  if (!vis || !n_out || (cap > 0 && !out) || (stats_cap > 0 && !stats))
    return fail(RF_ERR_INVALID_ARG, "bad periodicity-search arguments");
  if (nint < 1 || nint > p->max_nint) return fail(RF_ERR_SHAPE, "nint %d out of [1, %d]", nint, p->max_nint);
  if (L < 16 || L > 8192 || (L & (L - 1)) || L > nint)
    return fail(RF_ERR_INVALID_ARG, "L %d must be a power of two in [16, min(8192, nint)]", L);
  if (kmin < 1 || kmax < kmin || kmax > L / 2)
    return fail(RF_ERR_INVALID_ARG, "need 1 <= kmin <= kmax <= L/2 (kmin %d, kmax %d)", kmin, kmax);
  if (!(threshold > 0.0) || !std::isfinite(threshold)) return fail(RF_ERR_INVALID_ARG, "threshold must be > 0");
  BusyGuard bg(&p->busy);
  if (!bg.owned) return fail(RF_ERR_BUSY, "plan is in use by another call");
  DeviceGuard dg(p->device);
  if (!dg.ok) return fail(RF_ERR_CUDA, "cannot select device %d", p->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  *n_out = 0;
  if (n_stats) *n_stats = 0;
  rf_status s = ingest(p, vis, nint, st);
  if (s != RF_OK) return s;

  std::vector<int> dms;  // DM trials whose window and sweep fit in the segment
  for (int d = 0; d < p->ndm; ++d)
    if ((int64_t)p->max_delay[d] + L <= nint) dms.push_back(d);
  const int K = kmax - kmin + 1;
  const int kpad = (K + 31) / 32 * 32;
  const int B = p->shape.images_per_group;
  const int nkb = (K + B - 1) / B;
  const size_t nrows = (size_t)p->nbl * p->nchan;
  const size_t per_dm = 2 * nrows * kpad * sizeof(float2);
  const int ndms = (int)dms.size();
  const int nb_max = (int)std::max<size_t>(1, std::min<size_t>((size_t)std::max(ndms, 1), kPeriodicBudgetBytes / per_dm));
  const size_t npairs_total = (size_t)ndms * K;

  DeviceScratch sc;
  float2* d_per = nullptr;
  float2* d_twl = nullptr;
  int* d_dms = nullptr;
  int* d_zero = nullptr;
  int* d_ones = nullptr;
  int* d_lps = nullptr;
  unsigned long long* d_sdt = nullptr;
  Group* d_grp = nullptr;
  int4* d_pairs = nullptr;
  rf::DevPeriodic* d_pst = nullptr;
  rf::DevPeriodic* d_pc = nullptr;
  int* d_npc = nullptr;
  if ((s = sc.get(&d_per, (size_t)nb_max * per_dm / sizeof(float2))) != RF_OK || (s = sc.get(&d_twl, rf::fft_twiddle_len(L))) != RF_OK ||
      (s = sc.get(&d_dms, nb_max)) != RF_OK || (s = sc.get(&d_zero, p->nchan)) != RF_OK ||
      (s = sc.get(&d_ones, 2 * nb_max)) != RF_OK || (s = sc.get(&d_lps, 2 * nb_max)) != RF_OK ||
      (s = sc.get(&d_sdt, 2 * nb_max)) != RF_OK || (s = sc.get(&d_grp, (size_t)nb_max * nkb * 2)) != RF_OK ||
      (s = sc.get(&d_pairs, (size_t)nb_max * K)) != RF_OK || (s = sc.get(&d_pst, npairs_total)) != RF_OK ||
      (s = sc.get(&d_pc, npairs_total)) != RF_OK || (s = sc.get(&d_npc, 1)) != RF_OK)
    return s;
  {
    std::vector<float2> tw(rf::fft_twiddle_len(L));
    rf::fft_twiddle_table(L, tw.data());
    RF_CUDA(cudaMemcpyAsync(d_twl, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
    std::vector<int> ones(2 * nb_max, 1), lps(2 * nb_max, kpad);
    RF_CUDA(cudaMemcpyAsync(d_ones, ones.data(), ones.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    RF_CUDA(cudaMemcpyAsync(d_lps, lps.data(), lps.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    RF_CUDA(cudaMemsetAsync(d_zero, 0, p->nchan * sizeof(int), st));
    RF_CUDA(cudaMemsetAsync(d_npc, 0, sizeof(int), st));
    std::vector<unsigned long long> sdt(2 * nb_max);
    for (int q = 0; q < 2 * nb_max; ++q)
      sdt[q] = (unsigned long long)(uintptr_t)(d_per + (size_t)q * nrows * kpad);
    RF_CUDA(cudaMemcpyAsync(d_sdt, sdt.data(), sdt.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice, st));
  }
  // the search's gridding and column kernels, pointed at the transformed
  // series: "dt index" 2 j + q selects trial j's U (q = 0) or Q (q = 1)
  // series, delays are zero and "t'" is k - kmin
  rf::DevTables tbp = p->tb;
  tbp.delays = d_zero;
  tbp.dt_list = d_ones;
  tbp.sdt_ptr = d_sdt;
  tbp.sdt_lp = d_lps;
  const SegmentGeom g = geom(p, nint);
  SegmentGeom gp = g;
  gp.nint = K;
  gp.fp16 = false;   // the transformed series are FP32 whatever the storage
  gp.partial = false;  // every frequency index k - kmin < K of a group is present
  gp.idx32 = (uint64_t)nrows * kpad < (1ull << 32);

  for (int b0 = 0; b0 < ndms; b0 += nb_max) {
    const int nb = std::min(nb_max, ndms - b0);
    RF_CUDA(cudaMemcpyAsync(d_dms, dms.data() + b0, nb * sizeof(int), cudaMemcpyHostToDevice, st));
    RF_CUDA(rf::launch_period_dft(g, p->d_S, p->tb.delays, d_dms, nb, L, d_twl, kmin, K, kpad, d_per, st));
    // image list: per (trial j, block kb of up to B frequencies) a U group
    // then a Q group; a wave holds whole blocks so that each pair's two
    // images are in the same wave
    std::vector<Group> grp;
    std::vector<int4> pairs;
    struct PW { int g0, g1, i0, i1, p0, p1; };
    std::vector<PW> waves;
    PW w{0, 0, 0, 0, 0, 0};
    int nimg = 0;
    for (int j = 0; j < nb; ++j)
      for (int kb = 0; kb < nkb; ++kb) {
        const int n = std::min(B, K - kb * B);
        if ((nimg + 2 * n) - w.i0 > p->slots_max || ((int)grp.size() + 2) - w.g0 > p->gslots_max) {
          w.g1 = (int)grp.size();
          w.i1 = nimg;
          w.p1 = (int)pairs.size();
          waves.push_back(w);
          w = PW{w.g1, w.g1, nimg, nimg, w.p1, w.p1};
        }
        grp.push_back(Group{0, 2 * j, kb * B, n, nimg, {0, 0, 0}});
        grp.push_back(Group{0, 2 * j + 1, kb * B, n, nimg + n, {0, 0, 0}});
        for (int i = 0; i < n; ++i)
          pairs.push_back(make_int4(nimg + i - w.i0, nimg + n + i - w.i0, dms[b0 + j], kmin + kb * B + i));
        nimg += 2 * n;
      }
    w.g1 = (int)grp.size();
    w.i1 = nimg;
    w.p1 = (int)pairs.size();
    if (w.i1 > w.i0) waves.push_back(w);
    RF_CUDA(cudaMemcpyAsync(d_grp, grp.data(), grp.size() * sizeof(Group), cudaMemcpyHostToDevice, st));
    RF_CUDA(cudaMemcpyAsync(d_pairs, pairs.data(), pairs.size() * sizeof(int4), cudaMemcpyHostToDevice, st));
    const size_t pbase = (size_t)b0 * K;
    for (const PW& v : waves) {
      const int ng = v.g1 - v.g0;
      const int np = v.p1 - v.p0;
      RF_CUDA(rf::launch_grid_cells(gp, tbp, d_grp, v.g0, ng, p->d_cellbuf, st));
      RF_CUDA(rf::launch_colfft(gp, tbp, d_grp, v.g0, ng, v.i0, p->d_cellbuf, p->d_T, p->d_colsq, p->d_mean0, st));
      RF_CUDA(rf::launch_rowfft_power(gp, tbp, p->d_T, d_pairs + v.p0, np, p->d_partials,
                                      p->tmap_P.nbox > 0 ? &p->tmap_P : nullptr, p->d_err, st));
      RF_CUDA(rf::launch_finalize_power(gp, p->d_partials, p->d_colsq, p->d_mean0, d_pairs + v.p0, np,
                                        (int)(pbase + v.p0), (double)p->n_on, threshold, d_pst, d_pc, d_npc,
                                        (int)npairs_total, st));
    }
    // the host lists above are reused by the next batch
    RF_CUDA(cudaStreamSynchronize(st));
  }
  {
    int kerr = 0;
    RF_CUDA(cudaMemcpyAsync(&kerr, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    RF_CUDA(cudaStreamSynchronize(st));
    if (kerr) {
      cudaMemset(p->d_err, 0, sizeof(int));
      return fail(RF_ERR_TIMEOUT, "a periodicity row-pass tile copy did not complete within its wait limit");
    }
  }
  int npc = 0;
  RF_CUDA(cudaMemcpyAsync(&npc, d_npc, sizeof(int), cudaMemcpyDeviceToHost, st));
  RF_CUDA(cudaStreamSynchronize(st));
  npc = std::min(npc, (int)npairs_total);
  std::vector<rf::DevPeriodic> pc(npc), pst;
  if (npc > 0) RF_CUDA(cudaMemcpyAsync(pc.data(), d_pc, npc * sizeof(rf::DevPeriodic), cudaMemcpyDeviceToHost, st));
  if (stats && npairs_total > 0) {
    pst.resize(npairs_total);
    RF_CUDA(cudaMemcpyAsync(pst.data(), d_pst, npairs_total * sizeof(rf::DevPeriodic), cudaMemcpyDeviceToHost, st));
  }
  RF_CUDA(cudaStreamSynchronize(st));
  std::sort(pc.begin(), pc.end(), [](const rf::DevPeriodic& a, const rf::DevPeriodic& b) {
    return a.d != b.d ? a.d < b.d : a.k < b.k;
  });
  const int half = p->npix / 2;
  auto fill = [&](const rf::DevPeriodic& a, rf_periodic_candidate& o) {
    o.dm_idx = a.d;
    o.k = a.k;
    o.x = a.x;
    o.y = a.y;
    o.snr = a.snr;
    o.amplitude = a.amplitude;
    o.sigma = a.sigma;
    o.pad = 0.f;
    o.dm = p->dm[a.d];
    o.freq_hz = (double)a.k / ((double)L * p->inttime);
    o.l_rad = (double)(a.x - half) * p->cell;
    o.m_rad = (double)(a.y - half) * p->cell;
  };
  const size_t nw = std::min<size_t>(cap, pc.size());
  for (size_t k = 0; k < nw; ++k) fill(pc[k], out[k]);
  *n_out = pc.size();
  if (n_stats) *n_stats = npairs_total;
  if (stats) {
    const size_t ns = std::min(stats_cap, npairs_total);
    for (size_t k = 0; k < ns; ++k) fill(pst[k], stats[k]);
    if (npairs_total > stats_cap) return fail(RF_ERR_CAPACITY, "%zu stats, capacity %zu", npairs_total, stats_cap);
  }
  if (pc.size() > cap) return fail(RF_ERR_CAPACITY, "%zu candidates, capacity %zu", pc.size(), cap);
  return RF_OK;
}

rf_status rf_selftest_bounded_wait(int32_t device, int32_t polls, int32_t* gave_up) {
  if (!gave_up || polls < 1 || polls > (1 << 20)) return fail(RF_ERR_INVALID_ARG, "need gave_up and 1 <= polls <= 2^20");
  *gave_up = 0;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return fail(RF_ERR_NO_DEVICE, "no CUDA device");
  }
  if (device < 0 || device >= ndev) return fail(RF_ERR_INVALID_ARG, "device %d out of range", device);
  DeviceGuard dg(device);
  if (!dg.ok) return fail(RF_ERR_CUDA, "cannot select device %d", device);
  int* d = nullptr;
  RF_CUDA(cudaMalloc(&d, 2 * sizeof(int)));
  int h = 0;
  cudaError_t e = cudaMemset(d, 0, 2 * sizeof(int));
  if (e == cudaSuccess) e = rf::launch_wait_selftest(polls, d, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(RF_ERR_CUDA, "bounded-wait check: %s", cudaGetErrorString(e));
  *gave_up = h == 3 ? 1 : 0;  // both waits gave up
  return RF_OK;
}

rf_status rf_plan_set_form(rf_plan* plan, int32_t form) {
  if (!plan) return fail(RF_ERR_INVALID_ARG, "plan is NULL");
  if (form != RF_FORM_BATCHED && form != RF_FORM_PLAIN) return fail(RF_ERR_INVALID_ARG, "unknown form %d", form);
  plan->form = form;
  return RF_OK;
}

rf_status rf_plan_set_profiling(rf_plan* plan, int32_t enable) {
  if (!plan) return fail(RF_ERR_INVALID_ARG, "plan is NULL");
  BusyGuard bg(&plan->busy);
  if (!bg.owned) return fail(RF_ERR_BUSY, "plan is in use by another call");
  plan->prof.on = enable != 0;
  plan->prof.reset();
  return RF_OK;
}

rf_status rf_plan_get_profile(const rf_plan* plan, rf_kernel_profile* out, int32_t cap, int32_t* n) {
  if (!plan || !n || (cap > 0 && !out)) return fail(RF_ERR_INVALID_ARG, "NULL argument");
  *n = K_NKINDS;
  for (int k = 0; k < K_NKINDS && k < cap; ++k) {
    std::memset(out[k].name, 0, sizeof(out[k].name));
    std::strncpy(out[k].name, kKindNames[k], sizeof(out[k].name) - 1);
    out[k].launches = plan->prof.launches[k];
    out[k].total_ms = plan->prof.total_ms[k];
  }
  return RF_OK;
}

rf_status rf_plan_set_tuning(rf_plan* p, int32_t key, int64_t value) {
  if (!p) return fail(RF_ERR_INVALID_ARG, "plan is NULL");
  if (key == RF_TUNE_GRAPHS) {
    if (value != 0 && value != 1) return fail(RF_ERR_INVALID_ARG, "RF_TUNE_GRAPHS takes 0 or 1");
    BusyGuard bg(&p->busy);
    if (!bg.owned) return fail(RF_ERR_BUSY, "plan is in use by another call");
    DeviceGuard dg(p->device);
    p->use_graphs = value != 0;
    p->drop_graph();
    return RF_OK;
  }
  if (key == RF_TUNE_WIDE_INDEX) {
    if (value != 0 && value != 1) return fail(RF_ERR_INVALID_ARG, "RF_TUNE_WIDE_INDEX takes 0 or 1");
    BusyGuard bg(&p->busy);
    if (!bg.owned) return fail(RF_ERR_BUSY, "plan is in use by another call");
    DeviceGuard dg(p->device);
    p->wide_index = value != 0;
    p->drop_graph();  // captured launches carry the variant
    return RF_OK;
  }
  if (key == RF_TUNE_FUSED) {
    if (value != 0 && value != 1) return fail(RF_ERR_INVALID_ARG, "RF_TUNE_FUSED takes 0 or 1");
    BusyGuard bg(&p->busy);
    if (!bg.owned) return fail(RF_ERR_BUSY, "plan is in use by another call");
    DeviceGuard dg(p->device);
    p->fused = value != 0;
    p->cached_nint = -1;  // overlapped waves (half size) are built only without the fused pass
    p->drop_graph();
    return RF_OK;
  }
  if (key == RF_TUNE_OVERLAP) {
    if (value != 0 && value != 1) return fail(RF_ERR_INVALID_ARG, "RF_TUNE_OVERLAP takes 0 or 1");
    BusyGuard bg(&p->busy);
    if (!bg.owned) return fail(RF_ERR_BUSY, "plan is in use by another call");
    DeviceGuard dg(p->device);
    p->overlap = value != 0;
    p->cached_nint = -1;  // the waves' size depends on it
    p->drop_graph();
    return RF_OK;
  }
  if (key == RF_TUNE_RING) {
    if (value < 2 || value > 8) return fail(RF_ERR_INVALID_ARG, "RF_TUNE_RING takes 2 .. 8");
    if (p->host_only) return fail(RF_ERR_INVALID_ARG, "plan was created with RF_HOST_ONLY");
    BusyGuard bg(&p->busy);
    if (!bg.owned) return fail(RF_ERR_BUSY, "plan is in use by another call");
    DeviceGuard dg(p->device);
    if (p->chunk_images <= 0) {
      p->ring = (int)value;
      return RF_OK;
    }
    return alloc_ring(p, (int)value);
  }
  if (key != RF_TUNE_WAVE_IMAGES) return fail(RF_ERR_INVALID_ARG, "unknown tuning key %d", key);
  if (p->host_only) return fail(RF_ERR_INVALID_ARG, "plan was created with RF_HOST_ONLY");
  if (value < p->shape.images_per_group || value > 32768)
    return fail(RF_ERR_INVALID_ARG, "wave images %lld out of [%d, 32768]", (long long)value,
                p->shape.images_per_group);
  BusyGuard bg(&p->busy);
  if (!bg.owned) return fail(RF_ERR_BUSY, "plan is in use by another call");
  DeviceGuard dg(p->device);
  return alloc_wave_scratch(p, (int)value);
}

rf_status rf_plan_autotune(rf_plan* p, const void* vis, int32_t nint, void* stream, rf_tune_report* report) {
  if (!p) return fail(RF_ERR_INVALID_ARG, "plan is NULL");
  if (p->host_only) return fail(RF_ERR_INVALID_ARG, "plan was created with RF_HOST_ONLY");
  if (!vis) return fail(RF_ERR_INVALID_ARG, "vis is NULL");
  if (nint < 1 || nint > p->max_nint) return fail(RF_ERR_SHAPE, "nint %d out of [1, %d]", nint, p->max_nint);
  DeviceGuard dg(p->device);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t nimg = count_images(p, nint);
  const int B = p->shape.images_per_group;
  const size_t per_slot = (size_t)p->ncol * p->npix * sizeof(float2);
  size_t free_b = 0, total_b = 0;
  RF_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const size_t have = free_b / 2 + (size_t)p->slots_max * per_slot;  // the current scratch is reusable
  struct Cand {
    int wave, graphs, fused, ring, overlap;
  };
  std::vector<Cand> cands;
  auto fits = [&](int w) { return (size_t)std::max(w, B) * per_slot <= have; };
  const bool can_fuse = p->chunk_images > 0 && !(p->flags & RF_NOISE_CLIPPED);
  // waves whose column-FFT output fits the L2 cache (one to four groups), so
  // that the row pass may find it there instead of in HBM
  int l2 = 0;
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, p->device) != cudaSuccess) {
    cudaGetLastError();
    l2 = 0;
  }
  for (int w = B; w <= 4 * B && w < 256; w *= 2)
    if ((size_t)w * per_slot <= (size_t)l2 && fits(w) && w < nimg) cands.push_back({w, 1, 0, p->ring, 0});
  if (can_fuse) {
    for (int w : {2048, 8192}) {
      if (!fits(w)) continue;
      for (int ring : {2, 3, 4}) cands.push_back({w, 1, 1, ring, 0});
      cands.push_back({w, 1, 0, p->ring, 0});
      if (w / 2 >= B) cands.push_back({w, 1, 0, p->ring, 1});
      if (w >= nimg) break;
    }
  } else {
    for (int w : {256, 512, 1024, 2048, 4096, 8192}) {
      const int wc = std::max(w, B);
      if (!fits(wc)) continue;
      if (!cands.empty() && cands.back().wave >= nimg) break;
      cands.push_back({wc, 1, 0, p->ring, 0});
      cands.push_back({wc, 0, 0, p->ring, 0});
      if (wc >= 2048 && wc / 2 >= B && !(p->flags & RF_NOISE_CLIPPED)) cands.push_back({wc, 1, 0, p->ring, 1});
    }
  }
  if (cands.empty())
    cands.push_back({p->slots_max, p->use_graphs ? 1 : 0, p->fused ? 1 : 0, p->ring, p->overlap ? 1 : 0});

  // timing search: every (DM, dt) limited to its first nint/4 integrations
  const int span = nint >= 256 ? nint / 4 : 0;
  const bool prof_was = p->prof.on;
  p->prof.on = false;
  cudaEvent_t e0, e1;
  RF_CUDA(cudaEventCreate(&e0));
  RF_CUDA(cudaEventCreate(&e1));
  std::vector<rf_candidate> scratch_out(1);
  float best_ms = 1e30f;
  Cand best = cands[0];
  int ntried = 0;
  rf_status s = RF_OK;
  for (const Cand& c : cands) {
    {
      BusyGuard bg(&p->busy);
      if (!bg.owned) {
        s = fail(RF_ERR_BUSY, "plan is in use by another call");
        break;
      }
      if (p->slots_max != c.wave) s = alloc_wave_scratch(p, c.wave);
      if (s == RF_OK && c.fused && p->ring != c.ring) s = alloc_ring(p, c.ring);
      p->use_graphs = c.graphs != 0;
      p->fused = c.fused != 0;
      p->overlap = c.overlap != 0;
      p->cached_nint = -1;
      p->drop_graph();
    }
    if (s != RF_OK) break;
    size_t n_out = 0;
    rf_status r =
        search_impl(p, vis, nint, stream, scratch_out.data(), 0, &n_out, false, nullptr, 0, nullptr, span);
    if (r != RF_OK && r != RF_ERR_CAPACITY) {
      s = r;
      break;
    }
    cudaEventRecord(e0, st);
    r = search_impl(p, vis, nint, stream, scratch_out.data(), 0, &n_out, false, nullptr, 0, nullptr, span);
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    if (r != RF_OK && r != RF_ERR_CAPACITY) {
      s = r;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ntried < 16 && report) {
      report->tried_wave_images[ntried] = c.wave;
      report->tried_graphs[ntried] = c.graphs;
      report->tried_fused[ntried] = c.fused;
      report->tried_ring[ntried] = c.ring;
      report->tried_overlap[ntried] = c.overlap;
      report->tried_ms[ntried] = ms;
    }
    ++ntried;
    if (ms < best_ms) {
      best_ms = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  p->prof.on = prof_was;
  if (s != RF_OK) return s;
  {
    BusyGuard bg(&p->busy);
    if (p->slots_max != best.wave && (s = alloc_wave_scratch(p, best.wave)) != RF_OK) return s;
    if (best.fused && p->ring != best.ring && (s = alloc_ring(p, best.ring)) != RF_OK) return s;
    p->use_graphs = best.graphs != 0;
    p->fused = best.fused != 0;
    p->overlap = best.overlap != 0;
    p->cached_nint = -1;
    p->drop_graph();
  }
  if (report) {
    report->best_wave_images = best.wave;
    report->best_graphs = best.graphs;
    report->best_fused = best.fused;
    report->best_overlap = best.overlap;
    report->best_ring = p->ring;
    report->ntried = std::min(ntried, 16);
  }
  return RF_OK;
}

rf_status rf_plan_get_tuning(const rf_plan* p, int32_t key, int64_t* value) {
  if (!p || !value) return fail(RF_ERR_INVALID_ARG, "NULL argument");
  if (key == RF_TUNE_GRAPHS) {
    *value = p->use_graphs ? 1 : 0;
    return RF_OK;
  }
  if (key == RF_TUNE_WIDE_INDEX) {
    *value = p->wide_index ? 1 : 0;
    return RF_OK;
  }
  if (key == RF_TUNE_FUSED) {
    *value = p->fused ? 1 : 0;
    return RF_OK;
  }
  if (key == RF_TUNE_RING) {
    *value = p->ring;
    return RF_OK;
  }
  if (key == RF_TUNE_OVERLAP) {
    *value = p->overlap ? 1 : 0;
    return RF_OK;
  }
  if (key != RF_TUNE_WAVE_IMAGES) return fail(RF_ERR_INVALID_ARG, "unknown tuning key %d", key);
  *value = p->slots_max;
  return RF_OK;
}

rf_status rf_plan_get_info(const rf_plan* p, rf_plan_info* info) {
  if (!p || !info) return fail(RF_ERR_INVALID_ARG, "NULL argument");
  info->nbl = p->nbl;
  info->nchan = p->nchan;
  info->npix = p->npix;
  info->ndm = p->ndm;
  info->ndt = p->ndt;
  info->iu_max = p->iu_max;
  info->iv_max = p->iv_max;
  info->n_offgrid = p->n_offgrid;
  info->n_cells = (int32_t)p->n_cells;
  info->n_entries = (int32_t)p->ent.size();
  int mx = 0;
  for (int v : p->max_delay) mx = std::max(mx, v);
  info->max_delay = mx;
  info->images_per_group = p->shape.images_per_group;
  info->device_bytes = p->device_bytes;
  return RF_OK;
}

rf_status rf_plan_delays(const rf_plan* p, int32_t* out) {
  if (!p || !out) return fail(RF_ERR_INVALID_ARG, "NULL argument");
  std::memcpy(out, p->delays.data(), p->delays.size() * sizeof(int32_t));
  return RF_OK;
}

rf_status rf_plan_cells(const rf_plan* p, int32_t* iu, int32_t* iv, uint8_t* ongrid) {
  if (!p) return fail(RF_ERR_INVALID_ARG, "plan is NULL");
  if (iu) std::memcpy(iu, p->iu.data(), p->iu.size() * sizeof(int32_t));
  if (iv) std::memcpy(iv, p->iv.data(), p->iv.size() * sizeof(int32_t));
  if (ongrid) std::memcpy(ongrid, p->ongrid.data(), p->ongrid.size());
  return RF_OK;
}

rf_status rf_count_images(const rf_plan* p, int32_t nint, int64_t* n_images) {
  if (!p || !n_images) return fail(RF_ERR_INVALID_ARG, "NULL argument");
  if (nint < 0) return fail(RF_ERR_SHAPE, "nint must be >= 0");
  *n_images = count_images(p, nint);
  return RF_OK;
}

}  // extern "C"
