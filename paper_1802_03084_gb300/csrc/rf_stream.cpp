// rf_stream.cpp -- continuous search of a run of integrations cut into
// segments that overlap by the plan's longest dispersion sweep (Sec. 3.2).
//
// Segment k is the window of integrations [k stride, k stride + stride +
// overlap).  The raw visibilities of the window are kept on the device; when
// it is full the plan searches it with every (DM, dt) limited to
// t' < stride / dt, and the last `overlap` integrations are copied to the
// front of the other window, which the following pushes keep filling.  The
// device windows hold raw complex64 visibilities, so each segment is
// ingested (and, with RF_MEAN_SUBTRACT, mean-subtracted) on its own.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <deque>
#include <new>
#include <vector>

#include "realfast_gb300.h"
#include "rf_engine.h"

struct rf_stream {
  rf_plan* plan = nullptr;
  rf::PlanGeometry geo{};
  int stride = 0, overlap = 0, nseg = 0;
  uint32_t flags = 0;
  size_t per_int = 0;  // bytes of one raw integration
  unsigned char* win[2] = {nullptr, nullptr};
  int cur = 0;
  int fill = 0;
  int64_t pushed = 0;
  int64_t segments = 0;
  std::deque<rf_candidate> cands;
  std::deque<rf_image_stat> stats;
};

namespace {

rf_status fail(const char* msg, rf_status s = RF_ERR_INVALID_ARG) {
  rf::set_last_error(msg);
  return s;
}

struct DeviceScope {
  int prev = -1;
  bool ok = false;
  explicit DeviceScope(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && cudaSetDevice(dev) == cudaSuccess) ok = true;
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

rf_status cuda_fail(cudaError_t e) {
  rf::set_last_error(cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? RF_ERR_NO_MEMORY : RF_ERR_CUDA;
}

// Search `n` integrations of the current window (span 0: the plan's own
// edge rule) and queue the results with t_idx counted from the run start.
rf_status search_window(rf_stream* s, int n, int span, cudaStream_t st) {
  std::vector<rf_candidate> c;
  std::vector<rf_image_stat> im;
  const bool keep = (s->flags & RF_STREAM_KEEP_STATS) != 0;
  rf_status r = rf::search_span(s->plan, s->win[s->cur], n, span, st, &c, keep ? &im : nullptr);
  if (r != RF_OK) return r;
  const int64_t start = s->segments * (int64_t)s->stride;
  for (rf_candidate& x : c) {
    x.t_idx += (int32_t)(start / s->geo.dt[x.dt_idx]);
    s->cands.push_back(x);
  }
  for (rf_image_stat& x : im) {
    x.t_idx += (int32_t)(start / s->geo.dt[x.dt_idx]);
    s->stats.push_back(x);
  }
  return RF_OK;
}

}  // namespace

extern "C" {

rf_status rf_stream_create(rf_plan* plan, int32_t stride, uint32_t flags, rf_stream** out) {
  if (!out) return fail("rf_stream_create: out is NULL");
  *out = nullptr;
  if (!plan) return fail("rf_stream_create: plan is NULL");
  if (flags & ~RF_STREAM_KEEP_STATS) return fail("rf_stream_create: unknown flag bits");
  rf::PlanGeometry geo;
  rf_status r = rf::plan_geometry(plan, &geo);
  if (r != RF_OK) return r;
  if (geo.host_only) return fail("rf_stream_create: plan was created with RF_HOST_ONLY");
  if (stride < 1) return fail("rf_stream_create: stride must be >= 1");
  for (int dt : geo.dt)
    if (stride % dt != 0) return fail("rf_stream_create: stride must be a multiple of every dt of the plan");
  if ((int64_t)stride + geo.max_delay > geo.max_nint)
    return fail("rf_stream_create: stride + the longest sweep exceeds the plan's max_nint");
  DeviceScope ds(geo.device);
  if (!ds.ok) return fail("rf_stream_create: cannot select the plan's device", RF_ERR_CUDA);
  rf_stream* s = new (std::nothrow) rf_stream();
  if (!s) return fail("rf_stream_create: out of host memory", RF_ERR_NO_MEMORY);
  s->plan = plan;
  s->geo = geo;
  s->stride = stride;
  s->overlap = geo.max_delay;
  s->nseg = stride + geo.max_delay;
  s->flags = flags;
  s->per_int = (size_t)geo.nbl * geo.nchan * geo.npol * 8;
  for (int k = 0; k < 2; ++k) {
    cudaError_t e = cudaMalloc(&s->win[k], (size_t)s->nseg * s->per_int);
    if (e != cudaSuccess) {
      cudaGetLastError();
      rf_stream_destroy(s);
      return cuda_fail(e);
    }
  }
  *out = s;
  return RF_OK;
}

rf_status rf_stream_push(rf_stream* s, const void* vis, int32_t nint, void* stream, int32_t* n_segments) {
  if (n_segments) *n_segments = 0;
  if (!s) return fail("rf_stream_push: stream is NULL");
  if (nint < 0) return fail("rf_stream_push: nint < 0");
  if (nint > 0 && !vis) return fail("rf_stream_push: vis is NULL");
  DeviceScope ds(s->geo.device);
  if (!ds.ok) return fail("rf_stream_push: cannot select the plan's device", RF_ERR_CUDA);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const unsigned char* src = static_cast<const unsigned char*>(vis);
  int done = 0;
  int left = nint;
  while (left > 0) {
    const int take = std::min(left, s->nseg - s->fill);
    cudaError_t e = cudaMemcpyAsync(s->win[s->cur] + (size_t)s->fill * s->per_int, src, (size_t)take * s->per_int,
                                    cudaMemcpyDefault, st);
    if (e != cudaSuccess) return cuda_fail(e);
    src += (size_t)take * s->per_int;
    left -= take;
    s->fill += take;
    s->pushed += take;
    if (s->fill == s->nseg) {
      rf_status r = search_window(s, s->nseg, s->stride, st);
      if (r != RF_OK) return r;
      const int nxt = 1 - s->cur;
      if (s->overlap > 0) {
        e = cudaMemcpyAsync(s->win[nxt], s->win[s->cur] + (size_t)s->stride * s->per_int,
                            (size_t)s->overlap * s->per_int, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e);
      }
      s->cur = nxt;
      s->fill = s->overlap;
      s->segments += 1;
      done += 1;
    }
  }
  cudaError_t e = cudaStreamSynchronize(st);  // the caller may reuse vis on return
  if (e != cudaSuccess) return cuda_fail(e);
  if (n_segments) *n_segments = done;
  return RF_OK;
}

rf_status rf_stream_flush(rf_stream* s, void* stream, int32_t* n_segments) {
  if (n_segments) *n_segments = 0;
  if (!s) return fail("rf_stream_flush: stream is NULL");
  DeviceScope ds(s->geo.device);
  if (!ds.ok) return fail("rf_stream_flush: cannot select the plan's device", RF_ERR_CUDA);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (s->fill > 0) {
    rf_status r = search_window(s, s->fill, 0, st);
    if (r != RF_OK) return r;
    if (n_segments) *n_segments = 1;
  }
  s->cur = 0;
  s->fill = 0;
  s->pushed = 0;
  s->segments = 0;
  return RF_OK;
}

rf_status rf_stream_pop(rf_stream* s, rf_candidate* out, size_t cap, size_t* n_out) {
  if (!s || !n_out || (cap > 0 && !out)) return fail("rf_stream_pop: NULL argument");
  const size_t n = std::min(cap, s->cands.size());
  for (size_t k = 0; k < n; ++k) {
    out[k] = s->cands.front();
    s->cands.pop_front();
  }
  *n_out = n;
  return RF_OK;
}

rf_status rf_stream_pop_stats(rf_stream* s, rf_image_stat* out, size_t cap, size_t* n_out) {
  if (!s || !n_out || (cap > 0 && !out)) return fail("rf_stream_pop_stats: NULL argument");
  const size_t n = std::min(cap, s->stats.size());
  for (size_t k = 0; k < n; ++k) {
    out[k] = s->stats.front();
    s->stats.pop_front();
  }
  *n_out = n;
  return RF_OK;
}

rf_status rf_stream_get_info(const rf_stream* s, rf_stream_info* out) {
  if (!s || !out) return fail("rf_stream_get_info: NULL argument");
  out->stride = s->stride;
  out->overlap = s->overlap;
  out->segment_nint = s->nseg;
  out->fill = s->fill;
  out->pushed = s->pushed;
  out->segments = s->segments;
  out->pending_candidates = s->cands.size();
  out->pending_stats = s->stats.size();
  return RF_OK;
}

rf_status rf_stream_destroy(rf_stream* s) {
  if (!s) return RF_OK;
  DeviceScope ds(s->geo.device);
  for (int k = 0; k < 2; ++k)
    if (s->win[k]) cudaFree(s->win[k]);
  delete s;
  return RF_OK;
}

}  // extern "C"
