// C ABI of the wave library (include/wave.h): argument checking, workspace,
// host/device staging, sparse-point structures, the forward, adjoint and
// gradient sweeps and the checkpointed gradient.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "wave.h"
#include "wave_internal.h"

using namespace wave;

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct PointSetDev {
  bool valid = false;
  uint64_t key = 0;
  long long n = 0;
  int ncell = 0;
  std::string tag;  // workspace name prefix
  long long* base = nullptr;
  float* frac = nullptr;
  long long* cell = nullptr;
  int* rowptr = nullptr;
  int* pidx = nullptr;
  float* w = nullptr;
  float* coef = nullptr;
  std::vector<long long> cells_host;  // the cells, for the segment lists below
  // cells per CTA of the segmented step (CSR), for the decomposition seg_key
  uint64_t seg_key = 0;
  std::vector<int> seg_ptr_h, seg_list_h;
  int* seg_ptr = nullptr;
  int* seg_list = nullptr;
};

struct Pending {
  int kind;
  cudaEvent_t a, b;
};

}  // namespace

struct wave_context {
  int device = 0;
  size_t budget = 0;
  size_t held = 0;
  std::string err;
  EncodeTiledFn encode = nullptr;
  int* d_status = nullptr;
  int* h_status = nullptr;
  unsigned int* d_minmax = nullptr;
  unsigned int* h_minmax = nullptr;
  double* d_phi = nullptr;
  double* h_phi = nullptr;
  std::map<std::string, DevBuf> ws;
  PointSetDev pts[4];
  int pts_next = 0;
  bool profiling = false;
  std::vector<cudaEvent_t> ev_free;
  std::vector<Pending> pending;
  int64_t launches[WAVE_KERNEL_KINDS] = {};
  int64_t timed[WAVE_KERNEL_KINDS] = {};  // launches whose duration was taken with events
  double ms[WAVE_KERNEL_KINDS] = {};      // summed duration of the timed launches
  int ckpt_interval = 0;
  unsigned long long wait_ns = kWaitLimitNs;  // limit of the step kernels' progress waits
  int sm_count = 152;                         // multiprocessors of the device
  int time_block = 1;                         // time levels per pass of source-free forward modelling
  int col_segments = 1;                       // segmented plain step: 0 never, 1 where faster, 2 always (3D)
  bool withhold_next = false;                 // test hook: the next step launch issues no loads
  int last_plan[4] = {0, 0, 0, 0};  // fmt, buffer levels, parts per segment, segments
  // side stream and events that copy finished receiver rows to a pinned host
  // buffer while later time steps run (created on first use)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_rows = nullptr, ev_copied = nullptr, ev_input = nullptr;
  // page-locked staging of the request tables of batched session steps, and
  // the event after their last upload (the buffer is rewritten only after it)
  void* batch_host = nullptr;
  size_t batch_cap = 0;
  cudaEvent_t ev_batch = nullptr;
};

namespace {

int fail(wave_context* ctx, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf;
  return code;
}

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) {                                                                       \
      cudaGetLastError();                                                                          \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? WAVE_ERR_OUT_OF_MEMORY : WAVE_ERR_CUDA,  \
                  "%s failed: %s", #call, cudaGetErrorString(e_));                                 \
    }                                                                                              \
  } while (0)

#define TRY(expr)             \
  do {                        \
    int rc_ = (expr);         \
    if (rc_ != WAVE_OK) return rc_; \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int ws_get(wave_context* ctx, const std::string& name, size_t bytes, void** out) {
  bytes = round_up(std::max<size_t>(bytes, 256), 256);
  DevBuf& b = ctx->ws[name];
  if (b.bytes >= bytes) {
    *out = b.ptr;
    return WAVE_OK;
  }
  const size_t new_held = ctx->held - b.bytes + bytes;
  if (ctx->budget && new_held > ctx->budget)
    return fail(ctx, WAVE_ERR_OUT_OF_MEMORY, "workspace '%s' (%zu bytes) would exceed the budget of %zu bytes",
                name.c_str(), bytes, ctx->budget);
  if (b.ptr) {
    cudaFree(b.ptr);
    ctx->held -= b.bytes;
    b = DevBuf();
  }
  cudaError_t e = cudaMalloc(&b.ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b = DevBuf();
    return fail(ctx, WAVE_ERR_OUT_OF_MEMORY, "cudaMalloc of %zu bytes for '%s' failed: %s", bytes, name.c_str(),
                cudaGetErrorString(e));
  }
  b.bytes = bytes;
  ctx->held += bytes;
  *out = b.ptr;
  return WAVE_OK;
}

void ws_release(wave_context* ctx, const std::string& name) {
  auto it = ctx->ws.find(name);
  if (it == ctx->ws.end()) return;
  if (it->second.ptr) cudaFree(it->second.ptr);
  ctx->held -= it->second.bytes;
  ctx->ws.erase(it);
}

size_t ws_size(wave_context* ctx, const std::string& name) {
  auto it = ctx->ws.find(name);
  return it == ctx->ws.end() ? 0 : it->second.bytes;
}

int classify(wave_context* ctx, const void* p, bool* on_device) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *on_device = false;
    return WAVE_OK;
  }
  if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) {
    if (a.device != ctx->device)
      return fail(ctx, WAVE_ERR_INVALID_ARG, "device pointer belongs to device %d, context is on %d", a.device,
                  ctx->device);
    *on_device = true;
  } else {
    *on_device = false;
  }
  return WAVE_OK;
}

// Input array: device pointers are used in place, host arrays are copied into
// a named workspace buffer on `s`.
int stage_in(wave_context* ctx, const char* name, const void* p, size_t bytes, cudaStream_t s, const void** out) {
  if (bytes == 0) {
    *out = p;
    return WAVE_OK;
  }
  bool dev = false;
  TRY(classify(ctx, p, &dev));
  if (dev) {
    *out = p;
    return WAVE_OK;
  }
  void* d = nullptr;
  TRY(ws_get(ctx, std::string("in_") + name, bytes, &d));
  CK(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, s));
  *out = d;
  return WAVE_OK;
}

int ensure_copy_stream(wave_context* ctx) {
  if (!ctx->copy_stream) CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  if (!ctx->ev_rows) CK(cudaEventCreateWithFlags(&ctx->ev_rows, cudaEventDisableTiming));
  if (!ctx->ev_copied) CK(cudaEventCreateWithFlags(&ctx->ev_copied, cudaEventDisableTiming));
  if (!ctx->ev_input) CK(cudaEventCreateWithFlags(&ctx->ev_input, cudaEventDisableTiming));
  return WAVE_OK;
}

// Input first needed late in the call (observed data, adjoint sources): a
// page-locked host array is copied on the side stream, overlapping the work
// enqueued on `s` meanwhile, and *deferred tells the caller to make `s` wait
// on ctx->ev_input before the first use.  Other arrays go through stage_in.
int stage_in_deferred(wave_context* ctx, const char* name, const void* p, size_t bytes, cudaStream_t s,
                      const void** out, bool* deferred) {
  *deferred = false;
  bool dev = false;
  if (bytes > 0) TRY(classify(ctx, p, &dev));
  cudaPointerAttributes a;
  bool pinned = false;
  if (bytes > 0 && !dev) {
    if (cudaPointerGetAttributes(&a, p) == cudaSuccess) {
      pinned = a.type == cudaMemoryTypeHost;
    } else {
      cudaGetLastError();
    }
  }
  if (!pinned) return stage_in(ctx, name, p, bytes, s, out);
  TRY(ensure_copy_stream(ctx));
  void* d = nullptr;
  TRY(ws_get(ctx, std::string("in_") + name, bytes, &d));
  CK(cudaEventRecord(ctx->ev_input, s));  // after earlier work on s that may still read the buffer
  CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_input, 0));
  CK(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, ctx->copy_stream));
  CK(cudaEventRecord(ctx->ev_input, ctx->copy_stream));
  *out = d;
  *deferred = true;
  return WAVE_OK;
}

struct OutStage {
  void* user = nullptr;
  void* dev = nullptr;
  size_t bytes = 0;
  bool copy_back = false;
  bool pinned = false;  // the host buffer is page-locked: copies to it are asynchronous
};

int stage_out(wave_context* ctx, const char* name, void* p, size_t bytes, OutStage* o) {
  o->user = p;
  o->bytes = bytes;
  if (p == nullptr || bytes == 0) {
    o->dev = nullptr;
    return WAVE_OK;
  }
  bool dev = false;
  TRY(classify(ctx, p, &dev));
  if (dev) {
    o->dev = p;
    return WAVE_OK;
  }
  TRY(ws_get(ctx, std::string("out_") + name, bytes, &o->dev));
  o->copy_back = true;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) == cudaSuccess) {
    o->pinned = a.type == cudaMemoryTypeHost;
  } else {
    cudaGetLastError();
  }
  return WAVE_OK;
}

int finish_out(wave_context* ctx, const OutStage& o, cudaStream_t s) {
  if (o.copy_back) CK(cudaMemcpyAsync(o.user, o.dev, o.bytes, cudaMemcpyDeviceToHost, s));
  return WAVE_OK;
}

// ---------------------------------------------------------------- profiling
cudaEvent_t take_event(wave_context* ctx) {
  if (!ctx->ev_free.empty()) {
    cudaEvent_t e = ctx->ev_free.back();
    ctx->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

template <class F>
int launch(wave_context* ctx, int kind, cudaStream_t s, F&& f) {
  // with profiling on, every kProfileEvery-th launch of a kind is bracketed by
  // a pair of timing events (events on every launch add a few microseconds
  // of front-end work per kernel to the measured stream)
  constexpr int64_t kProfileEvery = 4;
  const int64_t index = ctx->launches[kind]++;
  cudaError_t e;
  if (ctx->profiling && index % kProfileEvery == 0) {
    Pending pd{kind, take_event(ctx), take_event(ctx)};
    cudaEventRecord(pd.a, s);
    e = f();
    cudaEventRecord(pd.b, s);
    ctx->pending.push_back(pd);
  } else {
    e = f();
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, WAVE_ERR_CUDA, "kernel launch failed: %s", cudaGetErrorString(e));
  }
  return WAVE_OK;
}

void collect_events(wave_context* ctx) {
  for (auto& pd : ctx->pending) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, pd.a, pd.b) == cudaSuccess) {
      ctx->ms[pd.kind] += t;
      ctx->timed[pd.kind]++;
    }
    cudaGetLastError();
    ctx->ev_free.push_back(pd.a);
    ctx->ev_free.push_back(pd.b);
  }
  ctx->pending.clear();
}

// ---------------------------------------------------------------- problem set-up
double fd_weight(int R, int j) {
  if (j == 0) {
    double s = 0;
    for (int k = 1; k <= R; ++k) s += 1.0 / (double(k) * k);
    return -2.0 * s;
  }
  // 2 (-1)^{j+1} (R!)^2 / (j^2 (R-j)! (R+j)!) = 2 (-1)^{j+1} / j^2 * prod_{i=1..j} (R-j+i)/(R+i)
  double r = 1.0;
  for (int i = 1; i <= j; ++i) r *= double(R - j + i) / double(R + i);
  return 2.0 * ((j % 2) ? 1.0 : -1.0) * r / (double(j) * j);
}

bool valid_order(int so) { return so >= 2 && so <= 16 && so % 2 == 0; }

double dt_limit(int ndim, const double* h, int so, double vmax) {
  const int R = so / 2;
  double abs_sum = std::fabs(fd_weight(R, 0));
  for (int j = 1; j <= R; ++j) abs_sum += 2.0 * std::fabs(fd_weight(R, j));
  double lam = 0;
  for (int d = 0; d < ndim; ++d) lam += abs_sum / (h[d] * h[d]);
  return 2.0 / (vmax * std::sqrt(lam));
}

struct Prob {
  int ndim = 0, so = 0, R = 0, nt = 0;
  float dt = 0;
  GridDims g{};
  double h[3] = {0, 0, 0};       // spacing per kernel axis
  double o[3] = {0, 0, 0};       // computational origin per kernel axis
  double lo[3] = {0, 0, 0};      // physical extent per kernel axis
  double hi[3] = {0, 0, 0};
  int n[3] = {1, 1, 1};          // computational points per kernel axis
  long long slot_elems = 0;      // NZ*NY*pitch
  long long phys_elems = 0;      // PZ*PY*PX
  long long dense_elems = 0;     // NZ*NY*NX
  int slabs_x = 0, slabs_y = 0;
  long long scale_elems = 0;     // slabs per level
  float em[3] = {0, 0, 0};       // eta_max/nbl^2 per kernel axis
  StepParams sp{};
  dim3 grid;
  // segmented plain step (3D): CTAs (0: z chunks only) and the start of each
  // CTA's run in the tile-major plane sequence (seg_ctas + 1 entries)
  int seg_ctas = 0;
  std::vector<long long> seg_runs;
  int tiles_x = 0, tiles_y = 0;
};

// Number of chunks the streamed axis (NZ planes) is cut into; the grid has
// `tiles` column tiles times that many CTAs, of which `slots` run at once.
// Rule, from measurements on 592^3 (ms per step launch for 1..9 chunks):
//   order 8:  0.707 0.610 0.551 0.529 0.557 0.547 0.535 0.530 0.528
//   order 16: 0.925 0.837 0.829 0.815 0.810 0.797 0.794 0.800 0.802
// at least 8 waves of CTAs (W = tiles c / slots >= 8), and among the counts
// from there up to twice that, the fullest last wave (W / ceil(W); the smaller
// count within 1 %): 9 chunks at order 8, 7 at order 16.  Chunks keep at least
// max(32, 4R) planes, since each CTA first loads the 2R planes of its z halo;
// where 8 waves are out of reach, the most chunks allowed are taken.
int choose_chunks(long long tiles, int NZ, int R, long long slots) {
  const int cmax = std::max(1, NZ / std::max(32, 4 * R));
  slots = std::max<long long>(1, slots);
  if (tiles * cmax < 8 * slots) return cmax;
  int lo = 1;
  while (tiles * lo < 8 * slots) ++lo;
  const int hi = std::min(cmax, 2 * lo);
  auto fill = [&](int c) {
    const double w = double(tiles * c) / double(slots);
    return w / std::ceil(w);
  };
  double best_fill = 0.0;
  for (int c = lo; c <= hi; ++c) best_fill = std::max(best_fill, fill(c));
  for (int c = lo; c <= hi; ++c)
    if (fill(c) >= best_fill - 0.01) return c;
  return lo;
}

// Column runs of the segmented plain step.  A CTA's cost is its planes plus
// kSegFill(R) plane times for each column segment it starts (the fill of its
// register queue: the 2R planes of the z halo, loaded a few at a time).  For a
// cost bound C the runs are cut greedily along the tile-major plane sequence
// (a run that reaches a column's end goes on in the next column if its budget
// allows, paying another fill); the smallest C that needs no more than `ctas`
// runs is found by bisection, so that runs crossing a column are shorter by
// about one fill.  Returns the run starts (runs + 1 entries) and C.
double seg_fill(int R) { return 4.0 + R; }

double seg_cut(long long tiles, int NZ, double fill, double C, std::vector<long long>* runs) {
  const long long total = tiles * NZ;
  long long g = 0, n = 0;
  double worst = 0;
  if (runs) runs->assign(1, 0);
  while (g < total) {
    double budget = C - fill;
    double cost = fill;
    long long end = g;
    while (true) {
      const long long e = NZ - end % NZ;  // planes left in this column
      if (budget < e) {
        const long long take = std::max<long long>(end == g ? 1 : 0, static_cast<long long>(budget));
        end += take;
        cost += static_cast<double>(take);
        break;
      }
      end += e;
      cost += static_cast<double>(e);
      budget -= static_cast<double>(e) + fill;
      if (end >= total || budget < 1.0) break;
      cost += fill;
    }
    end = std::min(end, total);
    worst = std::max(worst, cost);
    g = end;
    ++n;
    if (runs) runs->push_back(g);
  }
  return runs ? worst : static_cast<double>(n);
}

// Plans the segmented step for a grid of `tiles` columns of NZ planes whose
// z-chunk grid has `chunks` chunks per column and `slots` resident CTAs; true
// (and the run starts) where segments are taken.  The z-chunk grid runs in
// ceil(tiles c / slots) waves of NZ/c planes plus a fill; the runs cost the
// bound found above.  Segments are taken for grids of fewer than 4 waves where
// that is at least 3 % shorter (or always, with `force`), with at most one run
// per max(16, 2R) planes.  Larger grids keep the z chunks, whose concurrent
// CTAs share their halo planes in L2.
bool seg_plan(long long tiles, int NZ, int chunks, int R, long long slots, bool force, std::vector<long long>* runs) {
  const long long total = tiles * NZ;
  const long long min_run = std::max(16, 2 * R);
  const long long ctas = std::min(slots, std::max<long long>(1, total / min_run));
  const double fill = seg_fill(R);
  const double waves = std::ceil(double(tiles * chunks) / double(slots));
  if (!force && waves >= 4) return false;
  double lo = double(total) / double(ctas), hi = lo + 2.0 * fill + 1.0;
  while (seg_cut(tiles, NZ, fill, hi, nullptr) > double(ctas)) hi += fill;
  for (int it = 0; it < 50 && hi - lo > 0.25; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (seg_cut(tiles, NZ, fill, mid, nullptr) <= double(ctas)) hi = mid;
    else lo = mid;
  }
  const double t_seg = seg_cut(tiles, NZ, fill, hi, runs);
  const double t_chunks = waves * (double(NZ) / chunks + fill);
  return force || t_seg < 0.97 * t_chunks;
}

int prepare(wave_context* ctx, const wave_geometry* geom, float dt, int nt, int so, Prob* P) {
  if (!geom) return fail(ctx, WAVE_ERR_INVALID_ARG, "geometry is NULL");
  if (geom->ndim != 2 && geom->ndim != 3) return fail(ctx, WAVE_ERR_INVALID_ARG, "ndim must be 2 or 3");
  if (!valid_order(so)) return fail(ctx, WAVE_ERR_INVALID_ARG, "space_order must be even in [2, 16], got %d", so);
  if (nt < 2) return fail(ctx, WAVE_ERR_INVALID_ARG, "nt must be >= 2, got %d", nt);
  if (!(dt > 0.f) || !std::isfinite(dt)) return fail(ctx, WAVE_ERR_INVALID_ARG, "dt must be positive and finite");
  if (geom->nbl < 0 || geom->nbl > (1 << 20))
    return fail(ctx, WAVE_ERR_INVALID_ARG, "nbl = %d out of range [0, 2^20]", geom->nbl);
  if (geom->nbl > 0 && !(geom->sponge_vref > 0)) return fail(ctx, WAVE_ERR_INVALID_ARG, "sponge_vref must be > 0");
  const int nd = geom->ndim;
  double points = 1.0;  // computational points, in double so that no product overflows
  for (int d = 0; d < nd; ++d) {
    if (geom->shape[d] < 2 || geom->shape[d] > (1 << 20))
      return fail(ctx, WAVE_ERR_INVALID_ARG, "shape[%d] = %lld out of range [2, 2^20]", d, (long long)geom->shape[d]);
    if (!(geom->spacing[d] > 0) || !std::isfinite(geom->spacing[d]))
      return fail(ctx, WAVE_ERR_INVALID_ARG, "spacing[%d] must be positive", d);
    points *= double(geom->shape[d] + 2 * static_cast<long long>(geom->nbl) + 8);
  }
  // far beyond any device memory; the bound keeps every element count below
  // in 64-bit range
  if (points > 1099511627776.0)
    return fail(ctx, WAVE_ERR_INVALID_ARG, "computational grid of %.3g points exceeds 2^40", points);
  P->ndim = nd;
  P->so = so;
  P->R = so / 2;
  P->nt = nt;
  P->dt = dt;
  const int nbl = geom->nbl;
  GridDims& g = P->g;
  // kernel axes: 3D (x, y, z); 2D (x, depth, -)
  for (int a = 0; a < 3; ++a) {
    if (a < nd) {
      P->n[a] = static_cast<int>(geom->shape[a] + 2 * nbl);
      P->h[a] = geom->spacing[a];
      P->o[a] = geom->origin[a] - nbl * geom->spacing[a];
      P->lo[a] = geom->origin[a];
      P->hi[a] = geom->origin[a] + (geom->shape[a] - 1) * geom->spacing[a];
    } else {
      P->n[a] = 1;
      P->h[a] = 1.0;
    }
  }
  g.NX = P->n[0];
  g.NY = P->n[1];
  g.NZ = P->n[2];
  g.pitch = static_cast<int>(round_up(g.NX, 8));
  g.nblx = nbl;
  g.nbly = nbl;
  g.nblz = nd == 3 ? nbl : 0;
  g.PX = static_cast<int>(geom->shape[0]);
  g.PY = static_cast<int>(geom->shape[1]);
  g.PZ = nd == 3 ? static_cast<int>(geom->shape[2]) : 1;
  P->slot_elems = static_cast<long long>(g.NZ) * g.NY * g.pitch;
  P->phys_elems = static_cast<long long>(g.PZ) * g.PY * g.PX;
  P->dense_elems = static_cast<long long>(g.NZ) * g.NY * g.NX;
  P->slabs_x = (g.NX + kSlabX - 1) / kSlabX;
  P->slabs_y = (g.NY + kSlabY - 1) / kSlabY;
  P->scale_elems = static_cast<long long>(P->slabs_x) * P->slabs_y * g.NZ;
  for (int a = 0; a < nd; ++a) {
    if (nbl > 0) {
      const double emax = 3.0 * geom->sponge_vref * std::log(1000.0) / (2.0 * nbl * geom->spacing[a]);
      P->em[a] = static_cast<float>(emax / (double(nbl) * nbl));
    }
  }
  // stencil coefficients with 1/h^2 folded in
  StepParams& sp = P->sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.NX = g.NX;
  sp.NY = g.NY;
  sp.NZ = g.NZ;
  sp.pitch = g.pitch;
  sp.slot_elems = P->slot_elems;
  double inv_h2[3];
  for (int a = 0; a < 3; ++a) inv_h2[a] = (a < nd) ? 1.0 / (P->h[a] * P->h[a]) : 0.0;
  sp.c0 = static_cast<float>(fd_weight(P->R, 0) * (inv_h2[0] + inv_h2[1] + inv_h2[2]));
  for (int j = 1; j <= P->R; ++j) {
    const double w = fd_weight(P->R, j);
    sp.cx[j - 1] = static_cast<float>(w * inv_h2[0]);
    sp.cy[j - 1] = static_cast<float>(w * inv_h2[1]);
    sp.cz[j - 1] = static_cast<float>(w * inv_h2[2]);
  }
  bool equal = true;
  for (int j = 0; j < P->R; ++j)
    if (sp.cx[j] != sp.cy[j] || (nd == 3 && sp.cy[j] != sp.cz[j])) equal = false;
  sp.iso = iso_kernel(P->R, equal) ? 1 : 0;
  sp.nblx = g.nblx;
  sp.nbly = g.nbly;
  sp.nblz = g.nblz;
  sp.emx = P->em[0];
  sp.emy = P->em[1];
  sp.emz = P->em[2];
  sp.half_inv_dt = static_cast<float>(0.5 / double(dt));
  sp.inv_dt2 = static_cast<float>(1.0 / (double(dt) * dt));
  sp.slabs_x = P->slabs_x;
  sp.slabs_y = P->slabs_y;
  sp.status = ctx ? ctx->d_status : nullptr;  // no context: host-only queries
  sp.wait_ns = ctx ? ctx->wait_ns : kWaitLimitNs;
  // grid: x tiles, axis-1 tiles, chunks of the streamed axis
  const int tx = (g.NX + step_bx() - 1) / step_bx();
  const int ty = (g.NY + step_by(P->R, nd, sp.iso != 0) - 1) / step_by(P->R, nd, sp.iso != 0);
  int chunks = 1;
  if (nd == 3) {
    int layout[kStepLayoutMax];
    const int per_sm = step_layout(P->R, nd, MODE_PLAIN, sp.iso != 0, layout) > 8 ? layout[8] : 2;
    chunks = choose_chunks(static_cast<long long>(tx) * ty, g.NZ, P->R,
                           static_cast<long long>(ctx ? ctx->sm_count : 152) * per_sm);
  }
  sp.zchunk = (g.NZ + chunks - 1) / chunks;
  chunks = (g.NZ + sp.zchunk - 1) / sp.zchunk;
  if (ty > 65535 || chunks > 65535) return fail(ctx, WAVE_ERR_NOT_SUPPORTED, "grid too large for one launch");
  P->grid = dim3(tx, ty, chunks);
  P->tiles_x = tx;
  P->tiles_y = ty;
  if (nd == 3 && ctx && ctx->col_segments != 0) {
    int layout[kStepLayoutMax];
    const int per_sm = step_layout(P->R, nd, MODE_PLAIN, sp.iso != 0, layout) > 8 ? layout[8] : 2;
    const long long slots = static_cast<long long>(ctx->sm_count) * per_sm;
    if (seg_plan(static_cast<long long>(tx) * ty, g.NZ, chunks, P->R, slots, ctx->col_segments == 2, &P->seg_runs))
      P->seg_ctas = static_cast<int>(P->seg_runs.size()) - 1;
  }
  return WAVE_OK;
}

int make_map(wave_context* ctx, CUtensorMap* map, CUtensorMapDataType dtype, int rank, const void* base,
             const cuuint64_t* dims, const cuuint64_t* strides, const cuuint32_t* box) {
  cuuint32_t es[5] = {1, 1, 1, 1, 1};
  CUresult r = ctx->encode(map, dtype, rank, const_cast<void*>(base), dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(ctx, WAVE_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return WAVE_OK;
}

struct Work {
  float* fields = nullptr;  // 4 slots
  float* cm = nullptr;
  float* grad = nullptr;
  StepMaps maps;
};

// Model checks (positive, finite, dt within the stability limit) and the
// coefficient field cm = dt^2/m on the computational grid.
int setup_model(wave_context* ctx, Prob& P, const float* m_dev, float* cm, cudaStream_t s) {
  CK(cudaMemsetAsync(ctx->d_minmax, 0, 2 * sizeof(unsigned int), s));
  CK(cudaMemsetAsync(ctx->d_minmax, 0xff, sizeof(unsigned int), s));
  TRY(launch(ctx, WAVE_KERNEL_OTHER, s, [&] { return launch_minmax(m_dev, P.phys_elems, ctx->d_minmax, s); }));
  CK(cudaMemcpyAsync(ctx->h_minmax, ctx->d_minmax, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  float mmin, mmax;
  std::memcpy(&mmin, &ctx->h_minmax[0], 4);
  std::memcpy(&mmax, &ctx->h_minmax[1], 4);
  if (!(mmin > 0.f) || !std::isfinite(mmax) || ctx->h_minmax[0] == 0u)
    return fail(ctx, WAVE_ERR_INVALID_ARG, "model must be positive and finite (min %g, max %g)", mmin, mmax);
  const double vmax = 1.0 / std::sqrt(double(mmin));
  const double dtm = dt_limit(P.ndim, P.h, P.so, vmax);
  if (double(P.dt) > dtm)
    return fail(ctx, WAVE_ERR_UNSTABLE_DT, "dt = %g ms exceeds the stability limit %g ms (v_max = %g km/s)",
                double(P.dt), dtm, vmax);
  return launch(ctx, WAVE_KERNEL_OTHER, s, [&] {
    return launch_setup_cm(P.g, m_dev, cm, static_cast<float>(double(P.dt) * P.dt), s);
  });
}

// Tensor maps over a field buffer of `nslots` slots, the coefficient field and
// (optionally) the gradient.
int make_field_maps(wave_context* ctx, Prob& P, float* fields, int nslots, float* cm, float* grad, Work* W) {
  const GridDims& g = P.g;
  const int hx = step_hx(P.R);
  const int by = step_by(P.R, P.ndim, P.sp.iso != 0);
  const int bx = step_bx();
  {
    cuuint64_t dims[4] = {(cuuint64_t)g.NX, (cuuint64_t)g.NY, (cuuint64_t)g.NZ, (cuuint64_t)nslots};
    cuuint64_t str[3] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.pitch * g.NY * 4, (cuuint64_t)P.slot_elems * 4};
    cuuint32_t boxu[4] = {(cuuint32_t)(bx + 2 * hx), (cuuint32_t)(by + 2 * P.R), 1, 1};
    cuuint32_t boxp[4] = {(cuuint32_t)bx, (cuuint32_t)by, 1, 1};
    TRY(make_map(ctx, &W->maps.u, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, fields, dims, str, boxu));
    TRY(make_map(ctx, &W->maps.p, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, fields, dims, str, boxp));
  }
  {
    cuuint64_t dims[3] = {(cuuint64_t)g.NX, (cuuint64_t)g.NY, (cuuint64_t)g.NZ};
    cuuint64_t str[2] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.pitch * g.NY * 4};
    cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    TRY(make_map(ctx, &W->maps.cm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, cm, dims, str, box));
    if (grad) TRY(make_map(ctx, &W->maps.g, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, grad, dims, str, box));
    else W->maps.g = W->maps.cm;
  }
  W->maps.s = W->maps.p;
  W->fields = fields;
  W->cm = cm;
  W->grad = grad;
  P.sp.fields = fields;
  P.sp.status = ctx->d_status;
  return WAVE_OK;
}

// Field buffer (4 slots), coefficient field, optional gradient from the
// context workspace, with the model set-up and the tensor maps.
int prepare_fields(wave_context* ctx, Prob& P, const float* m_dev, cudaStream_t s, bool need_grad, Work* W) {
  void* p = nullptr;
  TRY(ws_get(ctx, "fields", 4 * P.slot_elems * sizeof(float), &p));
  float* fields = static_cast<float*>(p);
  TRY(ws_get(ctx, "cm", P.slot_elems * sizeof(float), &p));
  float* cm = static_cast<float*>(p);
  float* grad = nullptr;
  if (need_grad) {
    TRY(ws_get(ctx, "grad", P.slot_elems * sizeof(float), &p));
    grad = static_cast<float*>(p);
  }
  TRY(setup_model(ctx, P, m_dev, cm, s));
  return make_field_maps(ctx, P, fields, 4, cm, grad, W);
}

int snapshot_map(wave_context* ctx, Prob& P, int fmt, void* store, int levels, CUtensorMap* map) {
  const GridDims& g = P.g;
  const int es = fmt == 0 ? 4 : 2;
  cuuint64_t dims[4] = {(cuuint64_t)g.NX, (cuuint64_t)g.NY, (cuuint64_t)g.NZ, (cuuint64_t)levels};
  cuuint64_t str[3] = {(cuuint64_t)g.pitch * es, (cuuint64_t)g.pitch * g.NY * es, (cuuint64_t)P.slot_elems * es};
  cuuint32_t box[4] = {(cuuint32_t)step_bx(), (cuuint32_t)step_by(P.R, P.ndim, P.sp.iso != 0), 1, 1};
  const CUtensorMapDataType dt = fmt == 0 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                          : (fmt == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
  return make_map(ctx, map, dt, 4, store, dims, str, box);
}

// ---------------------------------------------------------------- sparse points
uint64_t fnv(uint64_t h, const void* p, size_t n) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= c[i];
    h *= 1099511628211ull;
  }
  return h;
}

// Host-side interpolation structures of one point set: per point the base
// cell and fractions (gather), and a CSR over unique cells (injection).
struct PointsHost {
  long long n = 0;
  uint64_t key = 0;
  std::vector<long long> base;
  std::vector<float> frac;
  std::vector<long long> cells;
  std::vector<int> rowptr, pidx;
  std::vector<float> wts;
};

// Coordinates of a point set on the host, and its cache key (coordinates and
// geometry).
int read_points(wave_context* ctx, Prob& P, const wave_points* pts, std::vector<float>* c, uint64_t* key_out) {
  if (!pts) return fail(ctx, WAVE_ERR_INVALID_ARG, "point set is NULL");
  const long long n = pts->n;
  // below 2^28 so that the 2^ndim corner entries of all points stay within
  // the 32-bit row pointers of the injection structure
  if (n < 0 || n >= (1LL << 28)) return fail(ctx, WAVE_ERR_INVALID_ARG, "point count %lld out of range [0, 2^28)", n);
  if (n > 0 && !pts->coords) return fail(ctx, WAVE_ERR_INVALID_ARG, "point coordinates are NULL");
  c->resize(static_cast<size_t>(n) * P.ndim);
  if (n > 0) {
    bool dev = false;
    TRY(classify(ctx, pts->coords, &dev));
    if (dev) CK(cudaMemcpy(c->data(), pts->coords, c->size() * sizeof(float), cudaMemcpyDeviceToHost));
    else std::memcpy(c->data(), pts->coords, c->size() * sizeof(float));
  }
  uint64_t key = 1469598103934665603ull;
  key = fnv(key, c->data(), c->size() * sizeof(float));
  key = fnv(key, &n, sizeof(n));
  key = fnv(key, &P.g, sizeof(P.g));
  key = fnv(key, P.h, sizeof(P.h));
  key = fnv(key, P.o, sizeof(P.o));
  key = fnv(key, P.lo, sizeof(P.lo));
  key = fnv(key, P.hi, sizeof(P.hi));
  *key_out = key;
  return WAVE_OK;
}

int build_points_from(wave_context* ctx, Prob& P, const std::vector<float>& c, uint64_t key, PointsHost* H) {
  const int nd = P.ndim;
  const long long n = static_cast<long long>(c.size() / nd);
  H->n = n;
  H->key = key;
  const GridDims& g = P.g;
  const long long sy = g.pitch, sz = static_cast<long long>(g.pitch) * g.NY;
  H->base.assign(static_cast<size_t>(n), 0);
  H->frac.assign(static_cast<size_t>(n) * 3, 0.f);
  struct Trip {
    long long cell;
    int p;
    float w;
  };
  const int C = 1 << nd;
  std::vector<Trip> trips;
  trips.reserve(static_cast<size_t>(n) * C);
  for (long long i = 0; i < n; ++i) {
    long long b = 0;
    double f[3] = {0, 0, 0};
    for (int a = 0; a < nd; ++a) {
      const double x = c[i * nd + a];
      if (!(x >= P.lo[a] && x <= P.hi[a]))
        return fail(ctx, WAVE_ERR_POINT_OUTSIDE, "point %lld axis %d coordinate %g outside [%g, %g]", i, a, x,
                    P.lo[a], P.hi[a]);
      const double t = (x - P.o[a]) / P.h[a];
      long long k = static_cast<long long>(std::floor(t));
      if (k >= P.n[a] - 1) k = P.n[a] - 2;
      if (k < 0) k = 0;
      double fr = t - double(k);
      fr = fr < 0 ? 0 : (fr > 1 ? 1 : fr);
      f[a] = fr;
      b += k * (a == 0 ? 1 : (a == 1 ? sy : sz));
    }
    H->base[i] = b;
    for (int a = 0; a < 3; ++a) H->frac[i * 3 + a] = static_cast<float>(f[a]);
    for (int cc = 0; cc < C; ++cc) {
      double w = 1.0;
      long long idx = b;
      for (int a = 0; a < nd; ++a) {
        const int bit = (cc >> a) & 1;
        w *= bit ? f[a] : 1.0 - f[a];
        idx += bit ? (a == 0 ? 1 : (a == 1 ? sy : sz)) : 0;
      }
      trips.push_back({idx, static_cast<int>(i), static_cast<float>(w)});
    }
  }
  std::sort(trips.begin(), trips.end(), [](const Trip& x, const Trip& y) {
    return x.cell < y.cell || (x.cell == y.cell && x.p < y.p);
  });
  H->cells.clear();
  H->rowptr.assign(1, 0);
  H->pidx.clear();
  H->wts.clear();
  for (size_t k = 0; k < trips.size(); ++k) {
    if (k == 0 || trips[k].cell != trips[k - 1].cell) {
      if (k > 0) H->rowptr.push_back(static_cast<int>(k));
      H->cells.push_back(trips[k].cell);
    }
    H->pidx.push_back(trips[k].p);
    H->wts.push_back(trips[k].w);
  }
  H->rowptr.push_back(static_cast<int>(trips.size()));
  if (H->cells.empty()) H->rowptr.assign(1, 0);
  return WAVE_OK;
}

int build_points_host(wave_context* ctx, Prob& P, const wave_points* pts, PointsHost* H) {
  std::vector<float> c;
  uint64_t key = 0;
  TRY(read_points(ctx, P, pts, &c, &key));
  return build_points_from(ctx, P, c, key, H);
}

// Device bytes of the uploaded structures of a point set (each array rounded
// like a workspace allocation).
size_t points_device_bytes(const PointsHost& H) {
  auto r = [](size_t b) { return round_up(std::max<size_t>(b, 256), 256); };
  return r(std::max<size_t>(1, H.base.size()) * 8) + r(std::max<size_t>(1, H.frac.size()) * 4) +
         r(std::max<size_t>(1, H.cells.size()) * 8) + r(H.rowptr.size() * 4) +
         r(std::max<size_t>(1, H.pidx.size()) * 4) + r(std::max<size_t>(1, H.wts.size()) * 4) +
         r(std::max<size_t>(1, H.cells.size()) * 4);
}

// Copy host structures into device arrays already placed in `e`.
int upload_points(wave_context* ctx, const PointsHost& H, PointSetDev& e, cudaStream_t s) {
  if (H.n > 0) {
    CK(cudaMemcpyAsync(e.base, H.base.data(), H.base.size() * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(e.frac, H.frac.data(), H.frac.size() * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(e.cell, H.cells.data(), H.cells.size() * 8, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(e.pidx, H.pidx.data(), H.pidx.size() * 4, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(e.w, H.wts.data(), H.wts.size() * 4, cudaMemcpyHostToDevice, s));
  }
  CK(cudaMemcpyAsync(e.rowptr, H.rowptr.data(), H.rowptr.size() * 4, cudaMemcpyHostToDevice, s));
  CK(cudaStreamSynchronize(s));  // the host vectors may go out of scope after this
  e.n = H.n;
  e.ncell = static_cast<int>(H.cells.size());
  e.key = H.key;
  e.cells_host = H.cells;
  e.seg_key = 0;
  e.valid = true;
  return WAVE_OK;
}

// Point structures for one call, cached in the context (keyed by coordinates
// and geometry) so repeated calls with the same points skip the build.
int prepare_points(wave_context* ctx, Prob& P, const wave_points* pts, cudaStream_t s, PointSetDev** out) {
  std::vector<float> c;
  uint64_t key = 0;
  TRY(read_points(ctx, P, pts, &c, &key));
  const long long n = pts->n;
  for (auto& e : ctx->pts) {
    if (e.valid && e.key == key && e.n == n) {
      *out = &e;
      return WAVE_OK;
    }
  }
  PointsHost H;
  TRY(build_points_from(ctx, P, c, key, &H));
  PointSetDev& e = ctx->pts[ctx->pts_next];
  ctx->pts_next = (ctx->pts_next + 1) % 4;
  e.valid = false;
  const int slot = static_cast<int>(&e - ctx->pts);
  e.tag = "pts" + std::to_string(slot) + "_";
  void* p = nullptr;
  TRY(ws_get(ctx, e.tag + "base", std::max<size_t>(1, H.base.size()) * 8, &p));
  e.base = static_cast<long long*>(p);
  TRY(ws_get(ctx, e.tag + "frac", std::max<size_t>(1, H.frac.size()) * 4, &p));
  e.frac = static_cast<float*>(p);
  TRY(ws_get(ctx, e.tag + "cell", std::max<size_t>(1, H.cells.size()) * 8, &p));
  e.cell = static_cast<long long*>(p);
  TRY(ws_get(ctx, e.tag + "rowptr", H.rowptr.size() * 4, &p));
  e.rowptr = static_cast<int*>(p);
  TRY(ws_get(ctx, e.tag + "pidx", std::max<size_t>(1, H.pidx.size()) * 4, &p));
  e.pidx = static_cast<int*>(p);
  TRY(ws_get(ctx, e.tag + "w", std::max<size_t>(1, H.wts.size()) * 4, &p));
  e.w = static_cast<float*>(p);
  TRY(ws_get(ctx, e.tag + "coef", std::max<size_t>(1, H.cells.size()) * 4, &p));
  e.coef = static_cast<float*>(p);
  TRY(upload_points(ctx, H, e, s));
  *out = &e;
  return WAVE_OK;
}

GatherSet gather_set(const Prob& P, const PointSetDev* ps) {
  GatherSet gs;
  gs.n = ps->n;
  gs.base = ps->base;
  gs.frac = ps->frac;
  gs.ndim = P.ndim;
  gs.sy = P.g.pitch;
  gs.sz = static_cast<long long>(P.g.pitch) * P.g.NY;
  return gs;
}

InjectSet inject_set(const PointSetDev* ps) {
  InjectSet is;
  is.n = ps->ncell;
  is.cell = ps->cell;
  is.rowptr = ps->rowptr;
  is.pidx = ps->pidx;
  is.w = ps->w;
  is.coef = ps->coef;
  return is;
}

int inject_coefficients(wave_context* ctx, Prob& P, Work& W, PointSetDev* ps, cudaStream_t s) {
  InjectSet is = inject_set(ps);
  return launch(ctx, WAVE_KERNEL_OTHER, s,
                [&] { return launch_inject_coef(is, P.g, W.cm, P.em, P.sp.half_inv_dt, s); });
}

// ---------------------------------------------------------------- sweeps
inline int fslot(int n) { return n & 1; }            // forward level n lives in slot n&1 (u^{-1} in slot 1)
inline int aslot(int j) { return 2 + (j & 1); }      // adjoint level j lives in slot 2 + (j&1)

float* slot_ptr(Work& W, const Prob& P, int slot) { return W.fields + slot * P.slot_elems; }

int step(wave_context* ctx, Prob& P, Work& W, int mode, int cur, int prev, cudaStream_t s) {
  P.sp.cur = cur;
  P.sp.prev = prev;
  const int kind = mode_is_grad(mode) ? WAVE_KERNEL_STEP_GRAD
                                      : (mode_is_snap(mode) ? WAVE_KERNEL_STEP_SNAP : WAVE_KERNEL_STEP);
  StepParams sp = P.sp;
  if (ctx->withhold_next) {
    sp.withhold = 1;
    ctx->withhold_next = false;
  }
  return launch(ctx, kind, s, [&] { return launch_step(P.R, P.ndim, mode, W.maps, sp, P.grid, s); });
}

struct SnapStore {
  int fmt = 0;            // 0 f32, 1 bf16, 2 f16
  int levels = 0;
  void* data = nullptr;
  float* scale = nullptr;
  CUtensorMap map;
  size_t level_bytes(const Prob& P) const { return static_cast<size_t>(P.slot_elems) * (fmt == 0 ? 4 : 2); }
  void* level(const Prob& P, int k) const { return static_cast<char*>(data) + level_bytes(P) * k; }
  float* level_scale(const Prob& P, int k) const { return scale ? scale + P.scale_elems * k : nullptr; }
};

int alloc_snapshots(wave_context* ctx, Prob& P, int fmt, int levels, SnapStore* S) {
  S->fmt = fmt;
  S->levels = levels;
  void* p = nullptr;
  TRY(ws_get(ctx, "snap", S->level_bytes(P) * levels, &p));
  S->data = p;
  if (fmt != 0) {
    TRY(ws_get(ctx, "snap_scale", static_cast<size_t>(P.scale_elems) * levels * 4, &p));
    S->scale = static_cast<float*>(p);
  } else {
    S->scale = nullptr;
  }
  return snapshot_map(ctx, P, fmt, S->data, levels, &S->map);
}

// Cells of an injection set per CTA of the segmented step: CSR over the
// CTAs (ptr, ctas + 1 entries) of indices into the set's cells (list).
void seg_cell_csr(const Prob& P, const std::vector<long long>& cells, std::vector<int>* ptr, std::vector<int>* list) {
  const int bx = step_bx(), by = step_by(P.R, P.ndim, P.sp.iso != 0);
  const int ctas = P.seg_ctas;
  std::vector<int> owner(cells.size());
  ptr->assign(static_cast<size_t>(ctas) + 1, 0);
  for (size_t k = 0; k < owner.size(); ++k) {
    const long long c = cells[k];
    const int x = static_cast<int>(c % P.g.pitch);
    const long long r = c / P.g.pitch;
    const int y = static_cast<int>(r % P.g.NY);
    const int z = static_cast<int>(r / P.g.NY);
    const long long col = static_cast<long long>(y / by) * P.tiles_x + x / bx;
    const long long g = col * P.g.NZ + z;
    owner[k] = static_cast<int>(std::upper_bound(P.seg_runs.begin(), P.seg_runs.end(), g) - P.seg_runs.begin()) - 1;
    (*ptr)[owner[k] + 1]++;
  }
  for (int b = 0; b < ctas; ++b) (*ptr)[b + 1] += (*ptr)[b];
  list->assign(std::max<size_t>(1, owner.size()), 0);
  std::vector<int> fill(ptr->begin(), ptr->end() - 1);
  for (size_t k = 0; k < owner.size(); ++k) (*list)[fill[owner[k]]++] = static_cast<int>(k);
}

// The same lists for a point set cached in the context (device copies in the
// context's workspace, kept on the point set for the decomposition they were
// made for).  Calls on a context run one after another and return after their
// stream completes, so its workspace serves them (resident sessions, whose
// launches stay queued on their own streams, never take the segmented step).
int seg_cell_lists(wave_context* ctx, const Prob& P, PointSetDev* ps, cudaStream_t s) {
  const int by = step_by(P.R, P.ndim, P.sp.iso != 0);
  uint64_t key = 1469598103934665603ull;
  const long long dims[6] = {P.seg_ctas, P.tiles_x, P.g.NZ, P.g.NY, P.g.pitch, by};
  key = fnv(key, dims, sizeof(dims));
  key = fnv(key, P.seg_runs.data(), P.seg_runs.size() * sizeof(long long));
  if (ps->seg_key == key && ps->seg_ptr) return WAVE_OK;
  seg_cell_csr(P, ps->cells_host, &ps->seg_ptr_h, &ps->seg_list_h);
  void* p = nullptr;
  TRY(ws_get(ctx, ps->tag + "segptr", ps->seg_ptr_h.size() * 4, &p));
  ps->seg_ptr = static_cast<int*>(p);
  TRY(ws_get(ctx, ps->tag + "seglist", ps->seg_list_h.size() * 4, &p));
  ps->seg_list = static_cast<int*>(p);
  // the host vectors stay with the point set until the copies are done
  CK(cudaMemcpyAsync(ps->seg_ptr, ps->seg_ptr_h.data(), ps->seg_ptr_h.size() * 4, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(ps->seg_list, ps->seg_list_h.data(), ps->seg_list_h.size() * 4, cudaMemcpyHostToDevice, s));
  ps->seg_key = key;
  return WAVE_OK;
}

// Plain forward steps n = n0 .. n1-1 by the segmented step: step n injects
// row n of q into level n+1 and samples receiver row n from level n (n > n0);
// row n1 is sampled after the last step.
int forward_steps_seg(wave_context* ctx, Prob& P, Work& W, int n0, int n1, const float* q, PointSetDev* src,
                      float* d, PointSetDev* rec, cudaStream_t s) {
  SegWork w{};
  w.inj = inject_set(src);
  void* runs = nullptr;
  TRY(ws_get(ctx, "seg_runs", P.seg_runs.size() * sizeof(long long), &runs));
  CK(cudaMemcpyAsync(runs, P.seg_runs.data(), P.seg_runs.size() * sizeof(long long), cudaMemcpyHostToDevice, s));
  w.run_start = static_cast<const long long*>(runs);
  if (w.inj.n > 0) {
    TRY(seg_cell_lists(ctx, P, src, s));
    w.inj_ptr = src->seg_ptr;
    w.inj_list = src->seg_list;
  }
  w.tiles_x = P.tiles_x;
  w.tiles_y = P.tiles_y;
  const bool sample = rec && rec->n > 0 && d;
  if (sample) w.rec = gather_set(P, rec);
  for (int n = n0; n < n1; ++n) {
    P.sp.cur = fslot(n);
    P.sp.prev = fslot(n - 1);
    StepParams sp = P.sp;
    if (ctx->withhold_next) {
      sp.withhold = 1;
      ctx->withhold_next = false;
    }
    w.inj_vals = w.inj.n > 0 ? q + static_cast<long long>(n) * src->n : nullptr;
    w.rec_out = sample && n > n0 ? d + static_cast<long long>(n) * rec->n : nullptr;
    TRY(launch(ctx, WAVE_KERNEL_STEP, s,
               [&] { return launch_step_seg(P.R, sp.iso != 0, W.maps, sp, w, P.seg_ctas, s); }));
  }
  if (sample && n1 > n0) {
    GatherSet grec = gather_set(P, rec);
    float* row = d + static_cast<long long>(n1) * rec->n;
    const float* level = slot_ptr(W, P, fslot(n1));
    TRY(launch(ctx, WAVE_KERNEL_SPARSE, s, [&] { return launch_gather(grec, level, row, s); }));
  }
  return WAVE_OK;
}

// Forward steps n = n0 .. n1-1 (each produces u^{n+1}); q rows injected; receiver
// rows gathered when d is given; centre levels n >= snap_from stored at
// level n - snap_base when S is given.
int forward_steps(wave_context* ctx, Prob& P, Work& W, int n0, int n1, const float* q, PointSetDev* src,
                  float* d, PointSetDev* rec, SnapStore* S, int snap_from, int snap_base, cudaStream_t s) {
  if (P.seg_ctas > 0 && (!S || n1 <= snap_from)) return forward_steps_seg(ctx, P, W, n0, n1, q, src, d, rec, s);
  InjectSet isrc = inject_set(src);
  GatherSet grec = rec ? gather_set(P, rec) : GatherSet{};
  for (int n = n0; n < n1; ++n) {
    int mode = MODE_PLAIN;
    if (S && n >= snap_from) {
      mode = S->fmt == 0 ? MODE_SNAP_F32 : (S->fmt == 1 ? MODE_SNAP_BF16 : MODE_SNAP_F16);
      P.sp.snap_out = S->level(P, n - snap_base);
      P.sp.scale_out = S->level_scale(P, n - snap_base);
    }
    TRY(step(ctx, P, W, mode, fslot(n), fslot(n - 1), s));
    float* out = slot_ptr(W, P, fslot(n + 1));
    if (isrc.n > 0) {
      const float* row = q + static_cast<long long>(n) * src->n;
      TRY(launch(ctx, WAVE_KERNEL_SPARSE, s, [&] { return launch_inject(isrc, row, out, s); }));
    }
    if (rec && rec->n > 0 && d) {
      float* row = d + static_cast<long long>(n + 1) * rec->n;
      TRY(launch(ctx, WAVE_KERNEL_SPARSE, s, [&] { return launch_gather(grec, out, row, s); }));
    }
  }
  return WAVE_OK;
}

// Source-free forward modelling with two time levels per pass (step2_kernel):
// levels rotate through the four field slots, since a pass reads level n with
// its halo and must write levels n+1 and n+2 elsewhere; an odd last level
// takes the single-level step.  Receiver rows of both output levels are
// gathered after each pass.  final_slot receives the slots of levels nt-2 and
// nt-1.
int forward_two_level(wave_context* ctx, Prob& P, Work& W, int nt, float* d, PointSetDev* rec, cudaStream_t s,
                      int* final_slot) {
  int ex, ey, uw, uh, bx, by;
  if (step2_box(P.R, &ex, &ey, &uw, &uh, &bx, &by) != 0)
    return fail(ctx, WAVE_ERR_NOT_SUPPORTED, "two-level pass needs space order 8");
  const GridDims& g = P.g;
  StepMaps maps;
  {
    cuuint64_t dims[4] = {(cuuint64_t)g.NX, (cuuint64_t)g.NY, (cuuint64_t)g.NZ, 4};
    cuuint64_t str[3] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.pitch * g.NY * 4, (cuuint64_t)P.slot_elems * 4};
    cuuint32_t boxu[4] = {(cuuint32_t)uw, (cuuint32_t)uh, 1, 1};
    cuuint32_t boxe[4] = {(cuuint32_t)ex, (cuuint32_t)ey, 1, 1};
    TRY(make_map(ctx, &maps.u, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, W.fields, dims, str, boxu));
    TRY(make_map(ctx, &maps.p, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, W.fields, dims, str, boxe));
    cuuint64_t dims3[3] = {(cuuint64_t)g.NX, (cuuint64_t)g.NY, (cuuint64_t)g.NZ};
    cuuint32_t box3[3] = {(cuuint32_t)ex, (cuuint32_t)ey, 1};
    TRY(make_map(ctx, &maps.cm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, W.cm, dims3, str, box3));
    maps.g = maps.cm;
    maps.s = maps.p;
  }
  const int tx = (g.NX + bx - 1) / bx, ty = (g.NY + by - 1) / by;
  int chunks = choose_chunks(static_cast<long long>(tx) * ty, g.NZ, 2 * P.R, ctx->sm_count);
  StepParams sp = P.sp;
  sp.zchunk = (g.NZ + chunks - 1) / chunks;
  chunks = (g.NZ + sp.zchunk - 1) / sp.zchunk;
  if (ty > 65535 || chunks > 65535) return fail(ctx, WAVE_ERR_NOT_SUPPORTED, "grid too large for one launch");
  const dim3 grid(tx, ty, chunks);
  GatherSet grec = rec ? gather_set(P, rec) : GatherSet{};
  auto gather = [&](int slot, int row) -> int {
    if (!rec || rec->n == 0 || !d) return WAVE_OK;
    float* out = d + static_cast<long long>(row) * rec->n;
    return launch(ctx, WAVE_KERNEL_SPARSE, s, [&] { return launch_gather(grec, slot_ptr(W, P, slot), out, s); });
  };
  int s_prev = fslot(-1), s_cur = fslot(0);
  int n = 0;
  for (; n + 2 <= nt - 1; n += 2) {
    int fr[2], k = 0;
    for (int sl = 0; sl < 4; ++sl)
      if (sl != s_prev && sl != s_cur) fr[k++] = sl;
    sp.cur = s_cur;
    sp.prev = s_prev;
    sp.out1 = fr[0];
    sp.out2 = fr[1];
    TRY(launch(ctx, WAVE_KERNEL_STEP, s, [&] { return launch_step2(P.R, maps, sp, grid, s); }));
    TRY(gather(fr[0], n + 1));
    TRY(gather(fr[1], n + 2));
    s_prev = fr[0];
    s_cur = fr[1];
  }
  if (n < nt - 1) {
    TRY(step(ctx, P, W, MODE_PLAIN, s_cur, s_prev, s));  // level n+1 overwrites level n-1
    TRY(gather(s_prev, n + 1));
    std::swap(s_prev, s_cur);
  }
  final_slot[0] = s_prev;
  final_slot[1] = s_cur;
  return WAVE_OK;
}

// Forward steps 0 .. nt-2 with the receiver rows copied to the caller's pinned
// host buffer in chunks on a side stream, overlapping the copies with the
// remaining steps; `s` waits for the last copy before the call returns.
int forward_steps_streamed(wave_context* ctx, Prob& P, Work& W, int nt, const float* q, PointSetDev* src,
                           PointSetDev* rec, const OutStage& dout, cudaStream_t s) {
  constexpr int kChunk = 128;  // time steps per copied block of rows
  TRY(ensure_copy_stream(ctx));
  const size_t row_bytes = static_cast<size_t>(rec->n) * sizeof(float);
  float* d = static_cast<float*>(dout.dev);
  long long rows_done = 0;
  for (int n0 = 0; n0 < nt - 1; n0 += kChunk) {
    const int n1 = std::min(n0 + kChunk, nt - 1);
    TRY(forward_steps(ctx, P, W, n0, n1, q, src, d, rec, nullptr, 0, 0, s));
    const long long rows_ready = n1 + 1;  // rows 0 .. n1 are final
    CK(cudaEventRecord(ctx->ev_rows, s));
    CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->ev_rows, 0));
    CK(cudaMemcpyAsync(static_cast<char*>(dout.user) + rows_done * row_bytes,
                       reinterpret_cast<const char*>(d) + rows_done * row_bytes,
                       static_cast<size_t>(rows_ready - rows_done) * row_bytes, cudaMemcpyDeviceToHost,
                       ctx->copy_stream));
    rows_done = rows_ready;
  }
  CK(cudaEventRecord(ctx->ev_copied, ctx->copy_stream));
  CK(cudaStreamWaitEvent(s, ctx->ev_copied, 0));
  return WAVE_OK;
}

int store_level(wave_context* ctx, Prob& P, Work& W, int slot, SnapStore* S, int k, cudaStream_t s) {
  return launch(ctx, WAVE_KERNEL_OTHER, s, [&] {
    return launch_snapshot_store(P.g, slot_ptr(W, P, slot), S->level(P, k), S->level_scale(P, k), S->fmt, P.slabs_x,
                                 P.slabs_y, s);
  });
}

// Adjoint-with-gradient iterations j = j1 .. j0 (descending); snapshot of u^j
// at level j - snap_base.
int adjoint_grad_steps(wave_context* ctx, Prob& P, Work& W, int j1, int j0, const float* y, PointSetDev* rec,
                       SnapStore* S, int snap_base, cudaStream_t s) {
  InjectSet irec = inject_set(rec);
  const int mode = S->fmt == 0 ? MODE_GRAD_F32 : (S->fmt == 1 ? MODE_GRAD_BF16 : MODE_GRAD_F16);
  for (int j = j1; j >= j0; --j) {
    const int lvl = j - snap_base;
    P.sp.snap_level = lvl;
    P.sp.scale_in = S->level_scale(P, lvl);
    P.sp.grad = W.grad;
    TRY(step(ctx, P, W, mode, aslot(j), aslot(j + 1), s));
    if (irec.n > 0) {
      float* out = slot_ptr(W, P, aslot(j - 1));
      const float* row = y + static_cast<long long>(j) * rec->n;
      const void* snap = S->level(P, lvl);
      const float* sc = S->level_scale(P, lvl);
      TRY(launch(ctx, WAVE_KERNEL_SPARSE, s, [&] {
        return launch_inject_grad(irec, row, out, W.grad, snap, S->fmt, sc, P.g, P.slabs_x, P.slabs_y, P.sp.inv_dt2,
                                  s);
      }));
    }
  }
  return WAVE_OK;
}

int begin_call(wave_context* ctx) {
  if (!ctx) return WAVE_ERR_INVALID_ARG;
  ctx->err.clear();
  return WAVE_OK;
}

// Synchronise, read the device status word, collect profiling events.
int end_call(wave_context* ctx, cudaStream_t s, int rc) {
  cudaError_t e1 = cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  collect_events(ctx);
  if (rc != WAVE_OK) {
    cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
    return rc;
  }
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    cudaError_t e = e2 != cudaSuccess ? e2 : e1;
    cudaGetLastError();
    return fail(ctx, WAVE_ERR_CUDA, "stream synchronisation failed: %s", cudaGetErrorString(e));
  }
  if (*ctx->h_status != kDevOk) {
    cudaMemsetAsync(ctx->d_status, 0, sizeof(int), s);
    cudaStreamSynchronize(s);
    return fail(ctx, WAVE_ERR_TIMEOUT, "a kernel gave up a bounded wait (device status %d)", *ctx->h_status);
  }
  return WAVE_OK;
}

int check_common(wave_context* ctx, const wave_geometry* geom, const float* m) {
  if (!ctx) return WAVE_ERR_INVALID_ARG;
  if (!geom || !m) return fail(ctx, WAVE_ERR_INVALID_ARG, "geometry or model is NULL");
  return WAVE_OK;
}

// ---------------------------------------------------------------- forward
int forward_impl(wave_context* ctx, const wave_geometry* geom, const float* m, const wave_points* src,
                 const float* q, const wave_points* rec, float* d_out, float dt, int nt, int so,
                 const float* u_init_prev, const float* u_init, float* u_final_prev, float* u_final, cudaStream_t s) {
  TRY(check_common(ctx, geom, m));
  Prob P;
  TRY(prepare(ctx, geom, dt, nt, so, &P));
  const long long ns = src ? src->n : 0, nr = rec ? rec->n : 0;
  if (ns > 0 && !q) return fail(ctx, WAVE_ERR_INVALID_ARG, "source traces are NULL");
  if (nr > 0 && !d_out) return fail(ctx, WAVE_ERR_INVALID_ARG, "receiver output is NULL");
  const void* mdev;
  TRY(stage_in(ctx, "m", m, P.phys_elems * 4, s, &mdev));
  const void* qdev = nullptr;
  if (ns > 0) TRY(stage_in(ctx, "q", q, static_cast<size_t>(nt) * ns * 4, s, &qdev));
  Work W;
  TRY(prepare_fields(ctx, P, static_cast<const float*>(mdev), s, false, &W));
  wave_points empty{0, nullptr};
  PointSetDev *S = nullptr, *Rr = nullptr;
  TRY(prepare_points(ctx, P, src ? src : &empty, s, &S));
  TRY(prepare_points(ctx, P, rec ? rec : &empty, s, &Rr));
  OutStage dout;
  TRY(stage_out(ctx, "d", d_out, static_cast<size_t>(nt) * nr * 4, &dout));
  TRY(inject_coefficients(ctx, P, W, S, s));
  // initial state
  for (int k = 0; k < 2; ++k) {
    const float* init = k == 0 ? u_init_prev : u_init;
    float* slot = slot_ptr(W, P, fslot(k - 1));
    if (init) {
      const void* dd;
      TRY(stage_in(ctx, k == 0 ? "u_init_prev" : "u_init", init, P.dense_elems * 4, s, &dd));
      CK(cudaMemsetAsync(slot, 0, P.slot_elems * 4, s));
      TRY(launch(ctx, WAVE_KERNEL_OTHER, s,
                 [&] { return launch_unpack_state(P.g, static_cast<const float*>(dd), slot, s); }));
    } else {
      CK(cudaMemsetAsync(slot, 0, P.slot_elems * 4, s));
    }
  }
  float* d = static_cast<float*>(dout.dev);
  if (nr > 0) {
    GatherSet grec = gather_set(P, Rr);
    TRY(launch(ctx, WAVE_KERNEL_SPARSE, s, [&] { return launch_gather(grec, slot_ptr(W, P, fslot(0)), d, s); }));
  }
  int final_slot[2] = {fslot(nt - 2), fslot(nt - 1)};
  if (ctx->time_block == 2 && P.ndim == 3 && P.R == 4 && ns == 0 && nt >= 3) {
    TRY(forward_two_level(ctx, P, W, nt, d, Rr, s, final_slot));
    TRY(finish_out(ctx, dout, s));
  } else if (dout.copy_back && dout.pinned) {
    TRY(forward_steps_streamed(ctx, P, W, nt, static_cast<const float*>(qdev), S, Rr, dout, s));
  } else {
    TRY(forward_steps(ctx, P, W, 0, nt - 1, static_cast<const float*>(qdev), S, d, Rr, nullptr, 0, 0, s));
    TRY(finish_out(ctx, dout, s));
  }
  for (int k = 0; k < 2; ++k) {
    float* fin = k == 0 ? u_final_prev : u_final;
    if (!fin) continue;
    OutStage o;
    TRY(stage_out(ctx, k == 0 ? "u_final_prev" : "u_final", fin, P.dense_elems * 4, &o));
    float* slot = slot_ptr(W, P, final_slot[k]);
    TRY(launch(ctx, WAVE_KERNEL_OTHER, s,
               [&] { return launch_pack_state(P.g, slot, static_cast<float*>(o.dev), s); }));
    TRY(finish_out(ctx, o, s));
  }
  return WAVE_OK;
}

// ---------------------------------------------------------------- adjoint
int adjoint_impl(wave_context* ctx, const wave_geometry* geom, const float* m, const wave_points* src,
                 const wave_points* rec, const float* y, float* q_out, float dt, int nt, int so, cudaStream_t s) {
  TRY(check_common(ctx, geom, m));
  Prob P;
  TRY(prepare(ctx, geom, dt, nt, so, &P));
  const long long ns = src ? src->n : 0, nr = rec ? rec->n : 0;
  if (nr > 0 && !y) return fail(ctx, WAVE_ERR_INVALID_ARG, "adjoint source traces are NULL");
  if (ns > 0 && !q_out) return fail(ctx, WAVE_ERR_INVALID_ARG, "adjoint output is NULL");
  const void* mdev;
  TRY(stage_in(ctx, "m", m, P.phys_elems * 4, s, &mdev));
  const void* ydev = nullptr;
  if (nr > 0) TRY(stage_in(ctx, "y", y, static_cast<size_t>(nt) * nr * 4, s, &ydev));
  Work W;
  TRY(prepare_fields(ctx, P, static_cast<const float*>(mdev), s, false, &W));
  wave_points empty{0, nullptr};
  PointSetDev *S = nullptr, *Rr = nullptr;
  TRY(prepare_points(ctx, P, src ? src : &empty, s, &S));
  TRY(prepare_points(ctx, P, rec ? rec : &empty, s, &Rr));
  OutStage qo;
  TRY(stage_out(ctx, "q_adj", q_out, static_cast<size_t>(nt) * ns * 4, &qo));
  TRY(inject_coefficients(ctx, P, W, Rr, s));
  CK(cudaMemsetAsync(slot_ptr(W, P, 2), 0, 2 * P.slot_elems * 4, s));
  float* qa = static_cast<float*>(qo.dev);
  if (ns > 0) CK(cudaMemsetAsync(qa + static_cast<long long>(nt - 1) * ns, 0, ns * 4, s));
  InjectSet irec = inject_set(Rr);
  GatherSet gsrc = gather_set(P, S);
  const float* yd = static_cast<const float*>(ydev);
  for (int j = nt - 1; j >= 1; --j) {
    TRY(step(ctx, P, W, MODE_PLAIN, aslot(j), aslot(j + 1), s));
    float* out = slot_ptr(W, P, aslot(j - 1));
    if (irec.n > 0) {
      const float* row = yd + static_cast<long long>(j) * nr;
      TRY(launch(ctx, WAVE_KERNEL_SPARSE, s, [&] { return launch_inject(irec, row, out, s); }));
    }
    if (ns > 0) {
      float* row = qa + static_cast<long long>(j - 1) * ns;
      TRY(launch(ctx, WAVE_KERNEL_SPARSE, s, [&] { return launch_gather(gsrc, out, row, s); }));
    }
  }
  TRY(finish_out(ctx, qo, s));
  return WAVE_OK;
}

// ---------------------------------------------------------------- Born modelling
// J dm: the background field u (with the Born source S written by its step)
// and the scattered field du (slots 2-3) advance together; S is corrected at
// the injected source cells like the imaging condition of the gradient.
int born_impl(wave_context* ctx, const wave_geometry* geom, const float* m, const float* dm, const wave_points* src,
              const float* q, const wave_points* rec, float* d_out, float dt, int nt, int so, cudaStream_t s) {
  TRY(check_common(ctx, geom, m));
  if (!dm) return fail(ctx, WAVE_ERR_INVALID_ARG, "model perturbation is NULL");
  Prob P;
  TRY(prepare(ctx, geom, dt, nt, so, &P));
  const long long ns = src ? src->n : 0, nr = rec ? rec->n : 0;
  if (ns > 0 && !q) return fail(ctx, WAVE_ERR_INVALID_ARG, "source traces are NULL");
  if (nr > 0 && !d_out) return fail(ctx, WAVE_ERR_INVALID_ARG, "receiver output is NULL");
  const void *mdev, *dmdev;
  TRY(stage_in(ctx, "m", m, P.phys_elems * 4, s, &mdev));
  TRY(stage_in(ctx, "dm", dm, P.phys_elems * 4, s, &dmdev));
  const void* qdev = nullptr;
  if (ns > 0) TRY(stage_in(ctx, "q", q, static_cast<size_t>(nt) * ns * 4, s, &qdev));
  Work W;
  TRY(prepare_fields(ctx, P, static_cast<const float*>(mdev), s, true, &W));  // W.grad holds S
  void* p = nullptr;
  TRY(ws_get(ctx, "dm_comp", P.slot_elems * 4, &p));
  float* dmc = static_cast<float*>(p);
  TRY(launch(ctx, WAVE_KERNEL_OTHER, s,
             [&] { return launch_pad_field(P.g, static_cast<const float*>(dmdev), dmc, s); }));
  StepMaps maps_born = W.maps, maps_src = W.maps;  // third tile: dm for the background, S for du
  {
    const GridDims& g = P.g;
    cuuint64_t dims[3] = {(cuuint64_t)g.NX, (cuuint64_t)g.NY, (cuuint64_t)g.NZ};
    cuuint64_t str[2] = {(cuuint64_t)g.pitch * 4, (cuuint64_t)g.pitch * g.NY * 4};
    cuuint32_t box[3] = {(cuuint32_t)step_bx(), (cuuint32_t)step_by(P.R, P.ndim, P.sp.iso != 0), 1};
    TRY(make_map(ctx, &maps_born.g, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, dmc, dims, str, box));
  }
  wave_points empty{0, nullptr};
  PointSetDev *Sp = nullptr, *Rr = nullptr;
  TRY(prepare_points(ctx, P, src ? src : &empty, s, &Sp));
  TRY(prepare_points(ctx, P, rec ? rec : &empty, s, &Rr));
  OutStage dout;
  TRY(stage_out(ctx, "d_born", d_out, static_cast<size_t>(nt) * nr * 4, &dout));
  TRY(inject_coefficients(ctx, P, W, Sp, s));
  CK(cudaMemsetAsync(W.fields, 0, 4 * P.slot_elems * 4, s));
  CK(cudaMemsetAsync(W.grad, 0, P.slot_elems * 4, s));
  float* d = static_cast<float*>(dout.dev);
  if (nr > 0) CK(cudaMemsetAsync(d, 0, nr * 4, s));  // du^0 = 0
  InjectSet isrc = inject_set(Sp);
  GatherSet grec = gather_set(P, Rr);
  const float* qd = static_cast<const float*>(qdev);
  P.sp.grad = W.grad;
  for (int n = 0; n < nt - 1; ++n) {
    P.sp.cur = fslot(n);
    P.sp.prev = fslot(n - 1);
    TRY(launch(ctx, WAVE_KERNEL_STEP, s,
               [&] { return launch_step(P.R, P.ndim, MODE_BORN_SRC, maps_born, P.sp, P.grid, s); }));
    if (isrc.n > 0) {
      const float* row = qd + static_cast<long long>(n) * ns;
      float* out = slot_ptr(W, P, fslot(n + 1));
      TRY(launch(ctx, WAVE_KERNEL_SPARSE, s, [&] {
        return launch_inject_grad(isrc, row, out, W.grad, dmc, 0, nullptr, P.g, P.slabs_x, P.slabs_y,
                                  P.sp.inv_dt2, s);
      }));
    }
    P.sp.cur = aslot(n);
    P.sp.prev = aslot(n - 1);
    TRY(launch(ctx, WAVE_KERNEL_STEP, s,
               [&] { return launch_step(P.R, P.ndim, MODE_SRC, maps_src, P.sp, P.grid, s); }));
    if (nr > 0) {
      float* row = d + static_cast<long long>(n + 1) * nr;
      const float* du = slot_ptr(W, P, aslot(n + 1));
      TRY(launch(ctx, WAVE_KERNEL_SPARSE, s, [&] { return launch_gather(grec, du, row, s); }));
    }
  }
  TRY(finish_out(ctx, dout, s));
  return WAVE_OK;
}

// ---------------------------------------------------------------- gradient
// Storage plan for the forward wavefield of Eq. 3.  A buffer of F snapshot
// levels first holds the last F levels (nt-F .. nt-1), stored during the
// forward sweep; the earlier levels [0, T0) are covered by segments of
// S = k*F levels that start at exact FP32 checkpoints (u^{k-1}, u^k).  In
// the reverse sweep each segment is rebuilt part by part, last part first:
// the part [A, A+F) is recomputed from the segment checkpoint into the same
// buffer, then swept by the adjoint.  k = 1 is classic two-level
// checkpointing, F = nt-1 is full storage; larger k trades recomputation
// ((k+1)/2 passes over the early part) for fewer checkpoints.
struct StoragePlan {
  int fmt = 0;   // 0 FP32, 1 BF16, 2 FP16
  int F = 0;     // levels in the snapshot buffer
  int k = 1;     // buffer-lengths per checkpointed segment
  int S = 0;     // segment length k*F
  int T0 = 1;    // first stored level of the tail
  int nseg = 0;  // checkpointed segments covering levels [0, T0)
};

// The sizing rule alone: lb bytes per buffer level, fb bytes per FP32 field
// (a checkpoint holds two), avail bytes for buffer and checkpoints.  Full
// storage unless ckpt; with ckpt, a fixed buffer of ckpt_interval levels if
// that is positive, else the smallest k (1, 2, 4 .. 64) for which some buffer
// fits, with the largest buffer that fits for that k.
int plan_levels(int nt, size_t lb, size_t fb, size_t avail, bool ckpt, int ckpt_interval, StoragePlan* plan) {
  int F = nt - 1, k = 1;
  if (ckpt) {
    if (ckpt_interval > 0) {
      F = std::min(ckpt_interval, nt - 1);
    } else {
      auto fits = [&](int FF, int kk) {
        const int T0 = nt - FF;
        const size_t nseg = static_cast<size_t>((T0 + kk * FF - 1) / (kk * FF));
        return static_cast<size_t>(FF) * lb + nseg * 2 * fb <= avail;
      };
      const int Fcap = static_cast<int>(std::min<size_t>(avail / lb, static_cast<size_t>(nt - 1)));
      F = 0;
      for (k = 1; k <= 64 && F == 0; k *= 2)
        for (int FF = Fcap; FF >= 1; --FF)
          if (fits(FF, k)) {
            F = FF;
            break;
          }
      k = F ? k / 2 : 1;
      if (F == 0) return WAVE_ERR_OUT_OF_MEMORY;
    }
  }
  plan->F = F;
  plan->k = k;
  plan->S = k * F;
  plan->T0 = nt - F;
  plan->nseg = plan->T0 > 1 ? (plan->T0 + plan->S - 1) / plan->S : 0;
  return WAVE_OK;
}

int plan_storage(wave_context* ctx, Prob& P, int mode, StoragePlan* plan) {
  if (mode < WAVE_SNAP_FULL_FP32 || mode > WAVE_SNAP_AUTO) return fail(ctx, WAVE_ERR_INVALID_ARG, "bad snap_mode %d", mode);
  const int nt = P.nt;
  const size_t fb = static_cast<size_t>(P.slot_elems) * 4;
  auto level_bytes = [&](int f) {
    return static_cast<size_t>(P.slot_elems) * (f == 0 ? 4 : 2) + (f == 0 ? 0 : static_cast<size_t>(P.scale_elems) * 4);
  };
  size_t avail;
  {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    cudaGetLastError();
    const size_t have = ws_size(ctx, "snap") + ws_size(ctx, "snap_scale") + ws_size(ctx, "ckpt");
    avail = fr + have;
    if (ctx->budget) {
      const size_t other = ctx->held - have;
      const size_t cap = ctx->budget > other ? ctx->budget - other : 0;
      avail = std::min(avail, cap);
    }
    avail = static_cast<size_t>(avail * 0.92);
  }
  int f = 0;
  bool ckpt = false;
  switch (mode) {
    case WAVE_SNAP_FULL_FP32: f = 0; break;
    case WAVE_SNAP_FULL_BF16: f = 1; break;
    case WAVE_SNAP_FULL_FP16: f = 2; break;
    case WAVE_SNAP_CHECKPOINT_FP32: f = 0; ckpt = true; break;
    case WAVE_SNAP_CHECKPOINT_BF16: f = 1; ckpt = true; break;
    case WAVE_SNAP_CHECKPOINT_FP16: f = 2; ckpt = true; break;
    case WAVE_SNAP_AUTO: f = 0; ckpt = level_bytes(0) * static_cast<size_t>(nt - 1) > avail; break;
  }
  plan->fmt = f;
  if (plan_levels(nt, level_bytes(f), fb, avail, ckpt, ctx->ckpt_interval, plan) != WAVE_OK)
    return fail(ctx, WAVE_ERR_OUT_OF_MEMORY, "the forward wavefield storage does not fit in memory");
  return WAVE_OK;
}

// zero_grad / fold: a multi-shot gradient accumulates every shot's imaging
// term into the same computational-grid buffer and folds once at the end.
int gradient_impl(wave_context* ctx, const wave_geometry* geom, const float* m, const wave_points* src,
                  const float* q, const wave_points* rec, const float* d_obs, const float* y_given,
                  float* grad_out, double* phi_out, float* resid_out, float* d_out, int snap_mode, float dt, int nt,
                  int so, cudaStream_t s, bool zero_grad = true, bool fold = true) {
  TRY(check_common(ctx, geom, m));
  if (!grad_out) return fail(ctx, WAVE_ERR_INVALID_ARG, "gradient output is NULL");
  Prob P;
  TRY(prepare(ctx, geom, dt, nt, so, &P));
  const long long ns = src ? src->n : 0, nr = rec ? rec->n : 0;
  if (ns > 0 && !q) return fail(ctx, WAVE_ERR_INVALID_ARG, "source traces are NULL");
  if (nr > 0 && !d_obs && !y_given) return fail(ctx, WAVE_ERR_INVALID_ARG, "observed data are NULL");
  const void* mdev;
  TRY(stage_in(ctx, "m", m, P.phys_elems * 4, s, &mdev));
  const void* qdev = nullptr;
  if (ns > 0) TRY(stage_in(ctx, "q", q, static_cast<size_t>(nt) * ns * 4, s, &qdev));
  const void* obs = nullptr;
  bool obs_deferred = false;
  if (nr > 0)
    TRY(stage_in_deferred(ctx, y_given ? "y" : "dobs", y_given ? y_given : d_obs, static_cast<size_t>(nt) * nr * 4, s,
                          &obs, &obs_deferred));
  Work W;
  TRY(prepare_fields(ctx, P, static_cast<const float*>(mdev), s, true, &W));
  wave_points empty{0, nullptr};
  PointSetDev *Sp = nullptr, *Rr = nullptr;
  TRY(prepare_points(ctx, P, src ? src : &empty, s, &Sp));
  TRY(prepare_points(ctx, P, rec ? rec : &empty, s, &Rr));
  TRY(inject_coefficients(ctx, P, W, Sp, s));
  TRY(inject_coefficients(ctx, P, W, Rr, s));
  OutStage gout, rout, dout;
  TRY(stage_out(ctx, "grad", grad_out, P.phys_elems * 4, &gout));
  TRY(stage_out(ctx, "resid", resid_out, static_cast<size_t>(nt) * nr * 4, &rout));
  TRY(stage_out(ctx, "dpred", d_out, static_cast<size_t>(nt) * nr * 4, &dout));
  void* p = nullptr;
  TRY(ws_get(ctx, "d_pred", std::max<size_t>(1, static_cast<size_t>(nt) * nr) * 4, &p));
  float* d = dout.dev ? static_cast<float*>(dout.dev) : static_cast<float*>(p);
  float* r = nullptr;
  if (y_given) {
    r = const_cast<float*>(static_cast<const float*>(obs));
  } else {
    TRY(ws_get(ctx, "resid_ws", std::max<size_t>(1, static_cast<size_t>(nt) * nr) * 4, &p));
    r = rout.dev ? static_cast<float*>(rout.dev) : static_cast<float*>(p);
  }
  const float* qd = static_cast<const float*>(qdev);
  // storage: a buffer of plan.F levels; checkpoints at the segment starts
  // (planned after every other buffer of the call is held)
  StoragePlan plan;
  TRY(plan_storage(ctx, P, snap_mode, &plan));
  ctx->last_plan[0] = plan.fmt;
  ctx->last_plan[1] = plan.F;
  ctx->last_plan[2] = plan.k;
  ctx->last_plan[3] = plan.nseg;
  SnapStore SS;
  const int T0 = plan.T0, S = plan.S, nseg = plan.nseg;
  float* ck = nullptr;
  if (nseg > 0) {
    TRY(ws_get(ctx, "ckpt", static_cast<size_t>(nseg) * 2 * P.slot_elems * 4, &p));
    ck = static_cast<float*>(p);
  }
  TRY(alloc_snapshots(ctx, P, plan.fmt, plan.F, &SS));
  W.maps.s = SS.map;
  // forward sweep: checkpoints before each segment start, the tail stored
  CK(cudaMemsetAsync(slot_ptr(W, P, 0), 0, 2 * P.slot_elems * 4, s));
  if (zero_grad) CK(cudaMemsetAsync(W.grad, 0, P.slot_elems * 4, s));
  if (nr > 0) {
    GatherSet grec = gather_set(P, Rr);
    TRY(launch(ctx, WAVE_KERNEL_SPARSE, s, [&] { return launch_gather(grec, slot_ptr(W, P, fslot(0)), d, s); }));
  }
  for (int seg = 0; seg < nseg; ++seg) {
    const int L0 = seg * S;
    const int L1 = std::min(L0 + S, T0);
    float* c0 = ck + static_cast<long long>(seg) * 2 * P.slot_elems;
    CK(cudaMemcpyAsync(c0, slot_ptr(W, P, fslot(L0 - 1)), P.slot_elems * 4, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(c0 + P.slot_elems, slot_ptr(W, P, fslot(L0)), P.slot_elems * 4, cudaMemcpyDeviceToDevice, s));
    TRY(forward_steps(ctx, P, W, L0, L1, qd, Sp, d, Rr, nullptr, 0, 0, s));
  }
  // steps n >= first computed step store the centre level n >= T0 at index n - T0
  const int n_first = nseg > 0 ? std::min(nseg * S, T0) : 0;
  TRY(forward_steps(ctx, P, W, n_first, nt - 1, qd, Sp, d, Rr, &SS, T0, T0, s));
  TRY(store_level(ctx, P, W, fslot(nt - 1), &SS, nt - 1 - T0, s));
  // the observed data (or adjoint sources) were uploaded during the forward sweep
  if (obs_deferred) CK(cudaStreamWaitEvent(s, ctx->ev_input, 0));
  // residual and objective
  if (nr > 0 && !y_given) {
    const long long n = static_cast<long long>(nt) * nr;
    const int nb = residual_blocks(n);
    TRY(ws_get(ctx, "partials", nb * sizeof(double), &p));
    double* part = static_cast<double*>(p);
    const float* dobs = static_cast<const float*>(obs);
    TRY(launch(ctx, WAVE_KERNEL_OTHER, s, [&] { return launch_residual(d, dobs, r, n, part, nb, s); }));
    TRY(launch(ctx, WAVE_KERNEL_OTHER, s, [&] { return launch_sum_partials(part, nb, ctx->d_phi, s); }));
  } else {
    CK(cudaMemsetAsync(ctx->d_phi, 0, sizeof(double), s));
  }
  // adjoint sweep with the imaging condition: the stored tail first ...
  CK(cudaMemsetAsync(slot_ptr(W, P, 2), 0, 2 * P.slot_elems * 4, s));
  TRY(adjoint_grad_steps(ctx, P, W, nt - 1, std::max(T0, 1), r, Rr, &SS, T0, s));
  // ... then the recomputed segments, last to first, each part by part
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int L0 = seg * S;
    const int L1 = std::min(L0 + S, T0);
    const float* c0 = ck + static_cast<long long>(seg) * 2 * P.slot_elems;
    for (int A = L0 + ((L1 - L0 - 1) / plan.F) * plan.F; A >= L0; A -= plan.F) {
      const int B = std::min(A + plan.F, L1);
      CK(cudaMemcpyAsync(slot_ptr(W, P, fslot(L0 - 1)), c0, P.slot_elems * 4, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(slot_ptr(W, P, fslot(L0)), c0 + P.slot_elems, P.slot_elems * 4, cudaMemcpyDeviceToDevice,
                         s));
      if (A > L0) TRY(forward_steps(ctx, P, W, L0, A, qd, Sp, nullptr, nullptr, nullptr, 0, 0, s));
      TRY(forward_steps(ctx, P, W, A, B - 1, qd, Sp, nullptr, nullptr, &SS, A, A, s));
      TRY(store_level(ctx, P, W, fslot(B - 1), &SS, B - 1 - A, s));
      const int jlo = std::max(A, 1);
      if (B - 1 >= jlo) TRY(adjoint_grad_steps(ctx, P, W, B - 1, jlo, r, Rr, &SS, A, s));
    }
  }
  if (fold) {
    TRY(launch(ctx, WAVE_KERNEL_OTHER, s,
               [&] { return launch_fold(P.g, W.grad, static_cast<float*>(gout.dev), s); }));
    TRY(finish_out(ctx, gout, s));
  }
  if (!y_given) TRY(finish_out(ctx, rout, s));
  TRY(finish_out(ctx, dout, s));
  CK(cudaMemcpyAsync(ctx->h_phi, ctx->d_phi, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (phi_out) *phi_out = *ctx->h_phi;
  return WAVE_OK;
}

// ---------------------------------------------------------------- sessions
// Device bytes a resident forward-modelling request holds: two wavefield
// slots, the coefficient field, staged model and source traces, receiver
// data, point structures, the step counter.
size_t session_bytes(const Prob& P, const PointsHost& hs, const PointsHost& hr, long long ns, long long nr) {
  auto r = [](size_t b) { return round_up(std::max<size_t>(b, 256), 256); };
  return r(2 * P.slot_elems * 4) + r(P.slot_elems * 4) + r(P.phys_elems * 4) + r(static_cast<size_t>(P.nt) * ns * 4) +
         r(static_cast<size_t>(P.nt) * nr * 4) + points_device_bytes(hs) + points_device_bytes(hr) + r(4);
}

// Resident sessions share the GPU with one another: the z chunks of one
// request's steps fill the waves another request leaves idle, and the column
// segments' cost model (one kernel alone on the GPU) does not apply.  Measured
// with the 600-request served stream: 11.9 shots/s with z chunks against 9.9 -
// 11.4 with segments.  So sessions keep the z-chunk grid, with the separate
// injection and sampling launches, for every step.
void session_grid(Prob* P) {
  P->seg_ctas = 0;
  P->seg_runs.clear();
}

}  // namespace

struct wave_session {
  wave_context* ctx = nullptr;
  cudaStream_t stream = nullptr;
  Prob P;
  Work W;
  PointSetDev src, rec;
  std::vector<std::pair<void*, size_t>> allocs;
  float* q = nullptr;
  float* d = nullptr;
  int* counter = nullptr;
  long long ns = 0, nr = 0;
  int next = 0;      // next time step to enqueue (steps are n = 0 .. nt-2)
  int chunk = 0;     // steps per captured graph (even)
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;
};

namespace {

int sess_alloc(wave_session* S, size_t bytes, void** out) {
  wave_context* ctx = S->ctx;
  bytes = round_up(std::max<size_t>(bytes, 256), 256);
  if (ctx->budget && ctx->held + bytes > ctx->budget)
    return fail(ctx, WAVE_ERR_OUT_OF_MEMORY, "request needs %zu more bytes than the budget allows", bytes);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, WAVE_ERR_OUT_OF_MEMORY, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  S->allocs.push_back({p, bytes});
  ctx->held += bytes;
  *out = p;
  return WAVE_OK;
}

void sess_free(wave_session* S) {
  for (auto& a : S->allocs) {
    cudaFree(a.first);
    S->ctx->held -= a.second;
  }
  S->allocs.clear();
}

int sess_points(wave_session* S, const PointsHost& H, PointSetDev* e) {
  void* p = nullptr;
  TRY(sess_alloc(S, std::max<size_t>(1, H.base.size()) * 8, &p));
  e->base = static_cast<long long*>(p);
  TRY(sess_alloc(S, std::max<size_t>(1, H.frac.size()) * 4, &p));
  e->frac = static_cast<float*>(p);
  TRY(sess_alloc(S, std::max<size_t>(1, H.cells.size()) * 8, &p));
  e->cell = static_cast<long long*>(p);
  TRY(sess_alloc(S, H.rowptr.size() * 4, &p));
  e->rowptr = static_cast<int*>(p);
  TRY(sess_alloc(S, std::max<size_t>(1, H.pidx.size()) * 4, &p));
  e->pidx = static_cast<int*>(p);
  TRY(sess_alloc(S, std::max<size_t>(1, H.wts.size()) * 4, &p));
  e->w = static_cast<float*>(p);
  TRY(sess_alloc(S, std::max<size_t>(1, H.cells.size()) * 4, &p));
  e->coef = static_cast<float*>(p);
  return upload_points(S->ctx, H, *e, S->stream);
}

// Kernels of `count` steps starting at an even step; the time rows of the
// sparse kernels come from the device counter so the same launches serve any
// even start (used while capturing the session's graph).
int enqueue_chunk_body(wave_session* S, int count, cudaStream_t s) {
  wave_context* ctx = S->ctx;
  Prob& P = S->P;
  InjectSet isrc = inject_set(&S->src);
  GatherSet grec = gather_set(P, &S->rec);
  for (int i = 0; i < count; ++i) {
    P.sp.cur = fslot(i);
    P.sp.prev = fslot(i - 1);
    cudaError_t e = launch_step(P.R, P.ndim, MODE_PLAIN, S->W.maps, P.sp, P.grid, s);
    if (e == cudaSuccess && isrc.n > 0)
      e = launch_inject_counter(isrc, S->q, S->ns, S->counter, i, slot_ptr(S->W, P, fslot(i + 1)), s);
    if (e == cudaSuccess && S->nr > 0)
      e = launch_gather_counter(grec, slot_ptr(S->W, P, fslot(i + 1)), S->d, S->counter, i + 1, s);
    if (e != cudaSuccess) return fail(ctx, WAVE_ERR_CUDA, "launch during capture failed: %s", cudaGetErrorString(e));
  }
  cudaError_t e = launch_counter_add(S->counter, count, s);
  if (e != cudaSuccess) return fail(ctx, WAVE_ERR_CUDA, "launch during capture failed: %s", cudaGetErrorString(e));
  return WAVE_OK;
}

// Capture one chunk on a private stream (the caller's stream may be the legacy
// default stream, which cannot be captured); the instantiated graph is then
// launched into the session's stream.
int session_capture(wave_session* S) {
  wave_context* ctx = S->ctx;
  cudaStream_t cs = nullptr;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  int rc = WAVE_OK;
  if (e != cudaSuccess) {
    cudaGetLastError();
    rc = fail(ctx, WAVE_ERR_CUDA, "stream capture failed to start: %s", cudaGetErrorString(e));
  } else {
    rc = enqueue_chunk_body(S, S->chunk, cs);
    e = cudaStreamEndCapture(cs, &graph);
    if (rc == WAVE_OK && e != cudaSuccess) {
      cudaGetLastError();
      rc = fail(ctx, WAVE_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(e));
    }
  }
  if (rc == WAVE_OK) {
    e = cudaGraphInstantiate(&S->exec, graph, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      rc = fail(ctx, WAVE_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
  }
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  return rc;
}

int session_create_impl(wave_context* ctx, wave_session* S, const wave_geometry* geom, const float* m,
                        const wave_points* src, const float* q, const wave_points* rec, float dt, int nt, int so) {
  TRY(check_common(ctx, geom, m));
  Prob& P = S->P;
  TRY(prepare(ctx, geom, dt, nt, so, &P));
  session_grid(&P);
  wave_points empty{0, nullptr};
  PointsHost hs, hr;
  TRY(build_points_host(ctx, P, src ? src : &empty, &hs));
  TRY(build_points_host(ctx, P, rec ? rec : &empty, &hr));
  S->ns = hs.n;
  S->nr = hr.n;
  if (S->ns > 0 && !q) return fail(ctx, WAVE_ERR_INVALID_ARG, "source traces are NULL");
  cudaStream_t s = S->stream;
  void* p = nullptr;
  TRY(sess_alloc(S, 2 * P.slot_elems * 4, &p));
  float* fields = static_cast<float*>(p);
  TRY(sess_alloc(S, P.slot_elems * 4, &p));
  float* cm = static_cast<float*>(p);
  TRY(sess_alloc(S, P.phys_elems * 4, &p));
  float* md = static_cast<float*>(p);
  TRY(sess_alloc(S, static_cast<size_t>(nt) * std::max<long long>(S->ns, 1) * 4, &p));
  S->q = static_cast<float*>(p);
  TRY(sess_alloc(S, static_cast<size_t>(nt) * std::max<long long>(S->nr, 1) * 4, &p));
  S->d = static_cast<float*>(p);
  TRY(sess_alloc(S, 4, &p));
  S->counter = static_cast<int*>(p);
  CK(cudaMemcpyAsync(md, m, P.phys_elems * 4, cudaMemcpyDefault, s));
  if (S->ns > 0) CK(cudaMemcpyAsync(S->q, q, static_cast<size_t>(nt) * S->ns * 4, cudaMemcpyDefault, s));
  TRY(sess_points(S, hs, &S->src));
  TRY(sess_points(S, hr, &S->rec));
  TRY(setup_model(ctx, P, md, cm, s));
  TRY(make_field_maps(ctx, P, fields, 2, cm, nullptr, &S->W));
  TRY(inject_coefficients(ctx, P, S->W, &S->src, s));
  CK(cudaMemsetAsync(fields, 0, 2 * P.slot_elems * 4, s));
  CK(cudaMemsetAsync(S->counter, 0, 4, s));
  if (S->nr > 0) {
    GatherSet grec = gather_set(P, &S->rec);
    TRY(launch(ctx, WAVE_KERNEL_SPARSE, s, [&] { return launch_gather(grec, slot_ptr(S->W, P, fslot(0)), S->d, s); }));
  }
  CK(cudaEventCreateWithFlags(&S->done, cudaEventDisableTiming));
  S->next = 0;
  if (S->chunk > 0 && nt - 1 >= S->chunk) TRY(session_capture(S));
  return WAVE_OK;
}

}  // namespace

// ============================================================================
// Public entry points
// ============================================================================
extern "C" {

int wave_context_create(wave_context** out, int device, size_t hbm_budget_bytes) {
  if (!out) return WAVE_ERR_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return WAVE_ERR_CUDA;
  }
  DeviceGuard guard(device);
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return WAVE_ERR_CUDA;
  if (prop.major * 10 + prop.minor != 103) return WAVE_ERR_NOT_SUPPORTED;  // kernels are built for sm_103a only
  wave_context* ctx = new wave_context();
  ctx->device = device;
  ctx->budget = hbm_budget_bytes;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || !fn) {
    cudaGetLastError();
    delete ctx;
    return WAVE_ERR_CUDA;
  }
  ctx->encode = reinterpret_cast<EncodeTiledFn>(fn);
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && sms > 0)
    ctx->sm_count = sms;
  cudaGetLastError();
  bool ok = cudaMalloc(&ctx->d_status, 16) == cudaSuccess && cudaMalloc(&ctx->d_minmax, 16) == cudaSuccess &&
            cudaMalloc(&ctx->d_phi, 16) == cudaSuccess &&
            cudaMallocHost(&ctx->h_status, 16) == cudaSuccess && cudaMallocHost(&ctx->h_minmax, 16) == cudaSuccess &&
            cudaMallocHost(&ctx->h_phi, 16) == cudaSuccess;
  if (ok) ok = cudaMemset(ctx->d_status, 0, 16) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    wave_context_destroy(ctx);
    return WAVE_ERR_CUDA;
  }
  *out = ctx;
  return WAVE_OK;
}

int wave_context_destroy(wave_context* ctx) {
  if (!ctx) return WAVE_OK;
  DeviceGuard guard(ctx->device);
  cudaDeviceSynchronize();
  for (auto& kv : ctx->ws)
    if (kv.second.ptr) cudaFree(kv.second.ptr);
  for (auto e : ctx->ev_free) cudaEventDestroy(e);
  for (auto& pd : ctx->pending) {
    cudaEventDestroy(pd.a);
    cudaEventDestroy(pd.b);
  }
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->d_minmax) cudaFree(ctx->d_minmax);
  if (ctx->d_phi) cudaFree(ctx->d_phi);
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  if (ctx->h_minmax) cudaFreeHost(ctx->h_minmax);
  if (ctx->h_phi) cudaFreeHost(ctx->h_phi);
  if (ctx->ev_rows) cudaEventDestroy(ctx->ev_rows);
  if (ctx->ev_copied) cudaEventDestroy(ctx->ev_copied);
  if (ctx->ev_input) cudaEventDestroy(ctx->ev_input);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->batch_host) cudaFreeHost(ctx->batch_host);
  if (ctx->ev_batch) cudaEventDestroy(ctx->ev_batch);
  cudaGetLastError();
  delete ctx;
  return WAVE_OK;
}

size_t wave_context_workspace_bytes(const wave_context* ctx) { return ctx ? ctx->held : 0; }

int wave_context_trim(wave_context* ctx) {
  if (!ctx) return WAVE_ERR_INVALID_ARG;
  DeviceGuard guard(ctx->device);
  cudaDeviceSynchronize();
  for (auto& kv : ctx->ws)
    if (kv.second.ptr) cudaFree(kv.second.ptr);
  ctx->ws.clear();
  ctx->held = 0;
  for (auto& e : ctx->pts) e.valid = false;
  return WAVE_OK;
}

int wave_context_set_checkpoint_interval(wave_context* ctx, int steps) {
  if (!ctx || steps < 0) return WAVE_ERR_INVALID_ARG;
  ctx->ckpt_interval = steps;
  return WAVE_OK;
}

int wave_context_set_wait_limit_ns(wave_context* ctx, uint64_t ns) {
  if (!ctx) return WAVE_ERR_INVALID_ARG;
  ctx->wait_ns = ns == 0 ? kWaitLimitNs : static_cast<unsigned long long>(ns);
  return WAVE_OK;
}

int wave_context_set_time_blocking(wave_context* ctx, int levels) {
  if (!ctx || (levels != 1 && levels != 2)) return WAVE_ERR_INVALID_ARG;
  ctx->time_block = levels;
  return WAVE_OK;
}

int wave_context_set_column_segments(wave_context* ctx, int mode) {
  if (!ctx) return WAVE_ERR_INVALID_ARG;
  if (mode < 0 || mode > 2) return fail(ctx, WAVE_ERR_INVALID_ARG, "column segment mode must be 0, 1 or 2");
  ctx->col_segments = mode;
  return WAVE_OK;
}

int wave_context_withhold_next_loads(wave_context* ctx) {
  if (!ctx) return WAVE_ERR_INVALID_ARG;
  ctx->withhold_next = true;
  return WAVE_OK;
}

const char* wave_error_string(int status) {
  switch (status) {
    case WAVE_OK: return "success";
    case WAVE_ERR_INVALID_ARG: return "invalid argument";
    case WAVE_ERR_POINT_OUTSIDE: return "point outside the physical domain";
    case WAVE_ERR_UNSTABLE_DT: return "time step above the stability limit";
    case WAVE_ERR_OUT_OF_MEMORY: return "out of device memory or workspace budget";
    case WAVE_ERR_CUDA: return "CUDA error";
    case WAVE_ERR_TIMEOUT: return "device-side wait timed out";
    case WAVE_ERR_NOT_SUPPORTED: return "not supported";
    default: return "unknown status";
  }
}

const char* wave_last_error(const wave_context* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int wave_forward_ex(wave_context* ctx, const wave_geometry* geom, const float* m, const wave_points* src,
                    const float* q, const wave_points* rec, float* d_out, float dt, int nt, int space_order,
                    const float* u_init_prev, const float* u_init, float* u_final_prev, float* u_final, void* stream) {
  TRY(begin_call(ctx));
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = forward_impl(ctx, geom, m, src, q, rec, d_out, dt, nt, space_order, u_init_prev, u_init, u_final_prev,
                        u_final, s);
  return end_call(ctx, s, rc);
}

int wave_forward(wave_context* ctx, const wave_geometry* geom, const float* m, const wave_points* src,
                 const float* q, const wave_points* rec, float* d_out, float dt, int nt, int space_order,
                 void* stream) {
  return wave_forward_ex(ctx, geom, m, src, q, rec, d_out, dt, nt, space_order, nullptr, nullptr, nullptr, nullptr,
                         stream);
}

int wave_adjoint(wave_context* ctx, const wave_geometry* geom, const float* m, const wave_points* src,
                 const wave_points* rec, const float* y, float* q_out, float dt, int nt, int space_order,
                 void* stream) {
  TRY(begin_call(ctx));
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = adjoint_impl(ctx, geom, m, src, rec, y, q_out, dt, nt, space_order, s);
  return end_call(ctx, s, rc);
}

int wave_gradient(wave_context* ctx, const wave_geometry* geom, const float* m, const wave_points* src,
                  const float* q, const wave_points* rec, const float* d_obs, float* grad_out, double* phi_out,
                  float* resid_out, int snap_mode, float dt, int nt, int space_order, void* stream) {
  TRY(begin_call(ctx));
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = gradient_impl(ctx, geom, m, src, q, rec, d_obs, nullptr, grad_out, phi_out, resid_out, nullptr, snap_mode,
                         dt, nt, space_order, s);
  return end_call(ctx, s, rc);
}

int wave_jacobian_adjoint(wave_context* ctx, const wave_geometry* geom, const float* m, const wave_points* src,
                          const float* q, const wave_points* rec, const float* y, float* grad_out, float* d_out,
                          int snap_mode, float dt, int nt, int space_order, void* stream) {
  TRY(begin_call(ctx));
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long nr = rec ? rec->n : 0;
  if (nr > 0 && !y) return end_call(ctx, s, fail(ctx, WAVE_ERR_INVALID_ARG, "adjoint source traces are NULL"));
  int rc = gradient_impl(ctx, geom, m, src, q, rec, nullptr, y, grad_out, nullptr, nullptr, d_out, snap_mode, dt, nt,
                         space_order, s);
  return end_call(ctx, s, rc);
}

int wave_gradient_shots(wave_context* ctx, const wave_geometry* geom, const float* m, int nshots,
                        const wave_points* srcs, const float* const* q, const wave_points* recs,
                        const float* const* d_obs, float* grad_out, double* phi_out, int snap_mode, float dt, int nt,
                        int space_order, void* stream) {
  TRY(begin_call(ctx));
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (nshots < 1 || !srcs || !recs || !q || !d_obs)
    return end_call(ctx, s, fail(ctx, WAVE_ERR_INVALID_ARG, "need nshots >= 1 and per-shot arrays"));
  double total = 0.0;
  int rc = WAVE_OK;
  for (int i = 0; i < nshots && rc == WAVE_OK; ++i) {
    double phi = 0.0;
    rc = gradient_impl(ctx, geom, m, &srcs[i], q[i], &recs[i], d_obs[i], nullptr, grad_out, &phi, nullptr, nullptr,
                       snap_mode, dt, nt, space_order, s, i == 0, i == nshots - 1);
    total += phi;
  }
  if (rc == WAVE_OK && phi_out) *phi_out = total;
  return end_call(ctx, s, rc);
}

int wave_born(wave_context* ctx, const wave_geometry* geom, const float* m, const float* dm, const wave_points* src,
              const float* q, const wave_points* rec, float* d_out, float dt, int nt, int space_order, void* stream) {
  TRY(begin_call(ctx));
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = born_impl(ctx, geom, m, dm, src, q, rec, d_out, dt, nt, space_order, s);
  return end_call(ctx, s, rc);
}

int wave_fd_weights(int space_order, double* w_out) {
  if (!valid_order(space_order) || !w_out) return WAVE_ERR_INVALID_ARG;
  const int R = space_order / 2;
  for (int j = 0; j <= R; ++j) w_out[j] = fd_weight(R, j);
  return WAVE_OK;
}

double wave_dt_max(int ndim, const double* spacing, int space_order, double v_max) {
  if ((ndim != 2 && ndim != 3) || !spacing || !valid_order(space_order) || !(v_max > 0)) return -1.0;
  for (int d = 0; d < ndim; ++d)
    if (!(spacing[d] > 0)) return -1.0;
  return dt_limit(ndim, spacing, space_order, v_max);
}

int wave_ricker(float* q_out, int nt, float dt, float f0, float t0) {
  if (!q_out || nt < 1 || !(dt > 0) || !(f0 > 0)) return WAVE_ERR_INVALID_ARG;
  std::vector<float> h(nt);
  const double pi = 3.14159265358979323846;
  for (int n = 0; n < nt; ++n) {
    const double a = pi * f0 * (n * double(dt) - t0);
    const double a2 = a * a;
    h[n] = static_cast<float>((1.0 - 2.0 * a2) * std::exp(-a2));
  }
  cudaPointerAttributes at;
  bool dev = cudaPointerGetAttributes(&at, q_out) == cudaSuccess &&
             (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  if (dev) {
    if (cudaMemcpy(q_out, h.data(), nt * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      return WAVE_ERR_CUDA;
    }
  } else {
    std::memcpy(q_out, h.data(), nt * sizeof(float));
  }
  return WAVE_OK;
}

int wave_step_kernel_layout(int space_order, int ndim, int kernel, int equal_spacing, int* out, int n_out,
                            int* n_values) {
  if (!valid_order(space_order) || (ndim != 2 && ndim != 3) || kernel < 0 || kernel >= MODE_COUNT || !out ||
      n_out < 1 || !n_values)
    return WAVE_ERR_INVALID_ARG;
  int v[kStepLayoutMax];
  const int n = step_layout(space_order / 2, ndim, kernel, equal_spacing != 0, v);
  if (n < 0 || n > kStepLayoutMax) return WAVE_ERR_INVALID_ARG;
  for (int i = 0; i < n && i < n_out; ++i) out[i] = v[i];
  *n_values = n;
  return WAVE_OK;
}

int wave_context_set_profiling(wave_context* ctx, int enable) {
  if (!ctx) return WAVE_ERR_INVALID_ARG;
  ctx->profiling = enable != 0;
  return WAVE_OK;
}

int wave_context_kernel_stats(wave_context* ctx, int kind, int64_t* launches, double* total_ms) {
  if (!ctx || kind >= WAVE_KERNEL_KINDS) return WAVE_ERR_INVALID_ARG;
  int64_t l = 0;
  double t = 0;
  for (int k = 0; k < WAVE_KERNEL_KINDS; ++k) {
    if (kind < 0 || k == kind) {
      l += ctx->launches[k];
      // the timed launches sample the kind: scale their mean to all launches
      if (ctx->timed[k] > 0) t += ctx->ms[k] * static_cast<double>(ctx->launches[k]) / ctx->timed[k];
    }
  }
  if (launches) *launches = l;
  if (total_ms) *total_ms = t;
  return WAVE_OK;
}

int wave_session_footprint(wave_context* ctx, const wave_geometry* geom, const wave_points* src,
                           const wave_points* rec, int nt, int space_order, size_t* bytes_out) {
  TRY(begin_call(ctx));
  if (!bytes_out) return fail(ctx, WAVE_ERR_INVALID_ARG, "bytes_out is NULL");
  Prob P;
  TRY(prepare(ctx, geom, 1.0f, nt, space_order, &P));
  wave_points empty{0, nullptr};
  PointsHost hs, hr;
  TRY(build_points_host(ctx, P, src ? src : &empty, &hs));
  TRY(build_points_host(ctx, P, rec ? rec : &empty, &hr));
  *bytes_out = session_bytes(P, hs, hr, std::max<long long>(hs.n, 1), std::max<long long>(hr.n, 1));
  return WAVE_OK;
}

int wave_session_create(wave_context* ctx, wave_session** out, const wave_geometry* geom, const float* m,
                        const wave_points* src, const float* q, const wave_points* rec, float dt, int nt,
                        int space_order, int graph_chunk, void* stream) {
  TRY(begin_call(ctx));
  if (!out) return fail(ctx, WAVE_ERR_INVALID_ARG, "session pointer is NULL");
  *out = nullptr;
  if (graph_chunk < 0 || graph_chunk % 2) return fail(ctx, WAVE_ERR_INVALID_ARG, "graph_chunk must be even and >= 0");
  DeviceGuard guard(ctx->device);
  wave_session* S = new wave_session();
  S->ctx = ctx;
  S->stream = static_cast<cudaStream_t>(stream);
  S->chunk = graph_chunk;
  int rc = session_create_impl(ctx, S, geom, m, src, q, rec, dt, nt, space_order);
  if (rc == WAVE_OK) {
    cudaError_t e = cudaStreamSynchronize(S->stream);
    if (e != cudaSuccess) rc = fail(ctx, WAVE_ERR_CUDA, "session set-up failed: %s", cudaGetErrorString(e));
  }
  if (rc != WAVE_OK) {
    cudaStreamSynchronize(S->stream);
    cudaGetLastError();
    if (S->exec) cudaGraphExecDestroy(S->exec);
    if (S->done) cudaEventDestroy(S->done);
    sess_free(S);
    delete S;
    return rc;
  }
  *out = S;
  return WAVE_OK;
}

int wave_session_advance(wave_session* S, int steps, int* steps_left) {
  if (!S) return WAVE_ERR_INVALID_ARG;
  wave_context* ctx = S->ctx;
  DeviceGuard guard(ctx->device);
  Prob& P = S->P;
  const int total = P.nt - 1;
  cudaStream_t s = S->stream;
  while (steps > 0 && S->next < total) {
    if (S->exec && S->next % S->chunk == 0 && total - S->next >= S->chunk) {
      CK(cudaGraphLaunch(S->exec, s));
      ctx->launches[WAVE_KERNEL_STEP] += S->chunk;
      ctx->launches[WAVE_KERNEL_SPARSE] += 2 * S->chunk;
      ctx->launches[WAVE_KERNEL_OTHER] += 1;
      S->next += S->chunk;
      steps -= S->chunk;
    } else {
      // steps that do not fill a whole captured chunk (the tail, or every
      // step when no graph was captured) run as ordinary launches
      const int stop = std::min(total, S->next + std::max(steps, 1));
      TRY(forward_steps(ctx, P, S->W, S->next, stop, S->q, &S->src, S->d, S->nr > 0 ? &S->rec : nullptr, nullptr,
                        0, 0, s));
      steps -= stop - S->next;
      S->next = stop;
    }
  }
  if (S->next >= total) CK(cudaEventRecord(S->done, s));
  if (steps_left) *steps_left = total - S->next;
  return WAVE_OK;
}

int wave_sessions_advance(wave_session* const* sessions, int n, int steps, void* stream) {
  if (n < 0 || steps < 0 || (n > 0 && !sessions)) return WAVE_ERR_INVALID_ARG;
  if (n == 0 || steps == 0) return WAVE_OK;
  if (!sessions[0]) return WAVE_ERR_INVALID_ARG;
  wave_context* ctx = sessions[0]->ctx;
  for (int i = 0; i < n; ++i)
    if (!sessions[i] || sessions[i]->ctx != ctx)
      return fail(ctx, WAVE_ERR_INVALID_ARG, "sessions must be non-NULL and share one context");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // this call's steps of every session, and its groups (radius, dimension,
  // spacing variant: one batched step launch per group and step)
  struct Item {
    wave_session* S;
    int n0, nlast;
  };
  std::vector<Item> items;
  int kmax = 0;
  for (int i = 0; i < n; ++i) {
    wave_session* S = sessions[i];
    const int total = S->P.nt - 1;
    const int take = std::min(steps, total - S->next);
    if (take <= 0) continue;
    items.push_back({S, S->next, S->next + take});
    kmax = std::max(kmax, take);
  }
  if (items.empty()) return WAVE_OK;
  std::map<int, std::vector<int>> groups;
  for (int i = 0; i < static_cast<int>(items.size()); ++i) {
    const Prob& P = items[i].S->P;
    groups[(P.R * 4 + P.ndim) * 2 + P.sp.iso].push_back(i);
  }
  const size_t step_bytes = sizeof(BatchStep) * items.size();
  const size_t sparse_off = round_up(step_bytes, 256);
  const size_t bytes = sparse_off + sizeof(BatchSparse) * items.size();
  if (ctx->ev_batch) CK(cudaEventSynchronize(ctx->ev_batch));  // the previous upload has read the staging
  if (bytes > ctx->batch_cap) {
    if (ctx->batch_host) cudaFreeHost(ctx->batch_host);
    ctx->batch_host = nullptr;
    ctx->batch_cap = 0;
    CK(cudaMallocHost(&ctx->batch_host, bytes));
    ctx->batch_cap = bytes;
  }
  if (!ctx->ev_batch) CK(cudaEventCreateWithFlags(&ctx->ev_batch, cudaEventDisableTiming));
  unsigned char* host = static_cast<unsigned char*>(ctx->batch_host);
  BatchStep* hstep = reinterpret_cast<BatchStep*>(host);
  BatchSparse* hsparse = reinterpret_cast<BatchSparse*>(host + sparse_off);
  struct Group {
    int R, ndim;
    bool iso;
    int first, count, ctas;
  };
  std::vector<Group> glist;
  int e = 0;
  bool any_src = false, any_rec = false;
  for (auto& kv : groups) {
    const Prob& P0 = items[kv.second[0]].S->P;
    Group gr{P0.R, P0.ndim, P0.sp.iso != 0, e, 0, 0};
    for (int i : kv.second) {
      const Item& it = items[i];
      const Prob& P = it.S->P;
      BatchStep& b = hstep[e++];
      b.maps = it.S->W.maps;
      b.p = P.sp;
      b.cta0 = gr.ctas;
      b.tiles_x = static_cast<int>(P.grid.x);
      b.tiles_y = static_cast<int>(P.grid.y);
      b.n0 = it.n0;
      b.nlast = it.nlast;
      gr.ctas += static_cast<int>(P.grid.x * P.grid.y * P.grid.z);
      gr.count++;
    }
    glist.push_back(gr);
  }
  int gctas = 0;
  for (int i = 0; i < static_cast<int>(items.size()); ++i) {
    wave_session* S = items[i].S;
    BatchSparse& b = hsparse[i];
    b.inj = inject_set(&S->src);
    b.q = S->q;
    b.ns = S->ns;
    b.gat = gather_set(S->P, &S->rec);
    b.d = S->d;
    b.fields = S->W.fields;
    b.slot_elems = S->P.slot_elems;
    b.n0 = items[i].n0;
    b.nlast = items[i].nlast;
    b.gcta0 = gctas;
    gctas += gather_batch_ctas(S->nr, S->P.ndim);
    any_src = any_src || S->src.ncell > 0;
    any_rec = any_rec || S->nr > 0;
  }
  void* dev = nullptr;
  TRY(ws_get(ctx, "batch_table", bytes, &dev));
  CK(cudaMemcpyAsync(dev, host, bytes, cudaMemcpyHostToDevice, s));
  CK(cudaEventRecord(ctx->ev_batch, s));
  const BatchStep* dstep = static_cast<const BatchStep*>(dev);
  const BatchSparse* dsparse = reinterpret_cast<const BatchSparse*>(static_cast<unsigned char*>(dev) + sparse_off);
  const int nitems = static_cast<int>(items.size());
  for (int k = 0; k < kmax; ++k) {
    for (const Group& gr : glist)
      TRY(launch(ctx, WAVE_KERNEL_STEP, s, [&] {
        return launch_step_batch(gr.R, gr.ndim, gr.iso, dstep + gr.first, gr.count, gr.ctas, k, s);
      }));
    if (any_src) TRY(launch(ctx, WAVE_KERNEL_SPARSE, s, [&] { return launch_inject_batch(dsparse, nitems, k, s); }));
    if (any_rec)
      TRY(launch(ctx, WAVE_KERNEL_SPARSE, s, [&] { return launch_gather_batch(dsparse, nitems, gctas, k, s); }));
  }
  for (const Item& it : items) {
    it.S->next = it.nlast;
    if (it.S->next >= it.S->P.nt - 1) CK(cudaEventRecord(it.S->done, s));
  }
  return WAVE_OK;
}

int wave_session_query(wave_session* S, int* done) {
  if (!S || !done) return WAVE_ERR_INVALID_ARG;
  *done = 0;
  if (S->next < S->P.nt - 1) return WAVE_OK;
  cudaError_t e = cudaEventQuery(S->done);
  if (e == cudaSuccess) *done = 1;
  else if (e != cudaErrorNotReady) {
    cudaGetLastError();
    return fail(S->ctx, WAVE_ERR_CUDA, "session query failed: %s", cudaGetErrorString(e));
  }
  return WAVE_OK;
}

int wave_session_read(wave_session* S, float* d_out) {
  if (!S) return WAVE_ERR_INVALID_ARG;
  wave_context* ctx = S->ctx;
  if (S->next < S->P.nt - 1) return fail(ctx, WAVE_ERR_INVALID_ARG, "session has steps left to enqueue");
  DeviceGuard guard(ctx->device);
  if (S->nr > 0 && !d_out) return fail(ctx, WAVE_ERR_INVALID_ARG, "output is NULL");
  // the last steps may have been enqueued on another stream (batched advance)
  CK(cudaStreamWaitEvent(S->stream, S->done, 0));
  if (S->nr > 0)
    CK(cudaMemcpyAsync(d_out, S->d, static_cast<size_t>(S->P.nt) * S->nr * 4, cudaMemcpyDefault, S->stream));
  CK(cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost, S->stream));
  CK(cudaStreamSynchronize(S->stream));
  if (*ctx->h_status != kDevOk) return fail(ctx, WAVE_ERR_TIMEOUT, "a kernel gave up a bounded wait");
  return WAVE_OK;
}

int wave_session_destroy(wave_session* S) {
  if (!S) return WAVE_OK;
  DeviceGuard guard(S->ctx->device);
  cudaStreamSynchronize(S->stream);
  if (S->done && S->next > 0) cudaEventSynchronize(S->done);  // steps enqueued on another stream
  if (S->exec) cudaGraphExecDestroy(S->exec);
  if (S->done) cudaEventDestroy(S->done);
  sess_free(S);
  cudaGetLastError();
  delete S;
  return WAVE_OK;
}

int wave_interpolation_operator(const wave_geometry* geom, const wave_points* pts, int64_t* index_out,
                                float* weight_out) {
  if (!geom || !pts || pts->n < 0 || pts->n >= (1LL << 28) || (pts->n > 0 && (!pts->coords || !index_out || !weight_out)))
    return WAVE_ERR_INVALID_ARG;
  Prob P;
  // the time step and order do not enter the interpolation
  TRY(prepare(nullptr, geom, 1.0f, 2, 2, &P));
  const int nd = P.ndim, C = 1 << nd;
  const long long n = pts->n;
  std::vector<float> c(pts->coords, pts->coords + n * nd);
  PointsHost H;
  TRY(build_points_from(nullptr, P, c, 0, &H));
  // read the operator back from the injection structure: rows are cells in
  // increasing order, so each point's entries arrive in corner order
  std::vector<int> filled(static_cast<size_t>(n), 0);
  const long long pitch = P.g.pitch, NX = P.g.NX, NY = P.g.NY;
  for (size_t r = 0; r + 1 < H.rowptr.size(); ++r) {
    const long long cell = H.cells[r];
    const long long x = cell % pitch, y = (cell / pitch) % NY, z = cell / (pitch * NY);
    const long long dense = (z * NY + y) * NX + x;
    for (int k = H.rowptr[r]; k < H.rowptr[r + 1]; ++k) {
      const int p = H.pidx[k];
      if (filled[p] >= C) return WAVE_ERR_INVALID_ARG;
      index_out[static_cast<long long>(p) * C + filled[p]] = dense;
      weight_out[static_cast<long long>(p) * C + filled[p]] = H.wts[k];
      ++filled[p];
    }
  }
  return WAVE_OK;
}

int wave_storage_plan_for(int nt, size_t level_bytes, size_t field_bytes, size_t avail_bytes, int checkpoint,
                          int checkpoint_interval, int* levels, int* parts, int* segments) {
  if (nt < 2 || level_bytes == 0 || checkpoint_interval < 0) return WAVE_ERR_INVALID_ARG;
  StoragePlan plan;
  const int rc = plan_levels(nt, level_bytes, field_bytes, avail_bytes, checkpoint != 0, checkpoint_interval, &plan);
  if (rc != WAVE_OK) return rc;
  if (levels) *levels = plan.F;
  if (parts) *parts = plan.k;
  if (segments) *segments = plan.nseg;
  return WAVE_OK;
}

int wave_column_runs_for(long long columns, int nz, int chunks, int space_order, long long slots, int force,
                         long long* run_start, int cap, int* n_runs) {
  if (columns < 1 || nz < 1 || chunks < 1 || slots < 1 || !valid_order(space_order) || !n_runs || cap < 0)
    return WAVE_ERR_INVALID_ARG;
  std::vector<long long> runs;
  *n_runs = 0;
  if (!seg_plan(columns, nz, chunks, space_order / 2, slots, force != 0, &runs)) return WAVE_OK;
  const int n = static_cast<int>(runs.size()) - 1;
  if (n + 1 > cap || !run_start) return WAVE_ERR_INVALID_ARG;
  std::copy(runs.begin(), runs.end(), run_start);
  *n_runs = n;
  return WAVE_OK;
}

int wave_z_chunks_for(long long columns, int nz, int space_order, long long slots, int* chunks) {
  if (columns < 1 || nz < 1 || slots < 1 || !valid_order(space_order) || !chunks) return WAVE_ERR_INVALID_ARG;
  *chunks = choose_chunks(columns, nz, space_order / 2, slots);
  return WAVE_OK;
}

int wave_context_storage_plan(const wave_context* ctx, int* levels, int* parts, int* segments) {
  if (!ctx) return WAVE_ERR_INVALID_ARG;
  if (levels) *levels = ctx->last_plan[1];
  if (parts) *parts = ctx->last_plan[2];
  if (segments) *segments = ctx->last_plan[3];
  return WAVE_OK;
}

size_t wave_context_budget_free(const wave_context* ctx) {
  if (!ctx || !ctx->budget) return 0;
  return ctx->budget > ctx->held ? ctx->budget - ctx->held : 0;
}

int wave_context_reset_stats(wave_context* ctx) {
  if (!ctx) return WAVE_ERR_INVALID_ARG;
  for (int k = 0; k < WAVE_KERNEL_KINDS; ++k) {
    ctx->launches[k] = 0;
    ctx->timed[k] = 0;
    ctx->ms[k] = 0;
  }
  return WAVE_OK;
}

}  // extern "C"
