// Host-side launch helpers of the stencil step (per radius, dimension and
// epilogue mode); included by the per-radius translation units.
#pragma once

#include <atomic>

#include "step_kernel.cuh"

namespace wave {

namespace dev {

// Batched plain step of the serving path: the CTAs of several resident
// requests (same radius, dimension and spacing variant) in one launch.  A CTA
// finds its request by a binary search over the first CTA of each request,
// copies the request's parameters behind the ring memory of the step body with
// the field slots of its step n = n0 + k, and runs the step body on its tile.
// Requests whose steps of this call are done (n >= nlast) return at once.
// The tensor maps are read from the table in device memory; the producer
// orders them for the tensor-map proxy before its first copy.
template <int R, int NDIM, bool ISO>
__global__ void __launch_bounds__(StepTraits<R, NDIM, ISO>::NTHREADS, (StepLayout<R, NDIM, MODE_PLAIN, ISO>::MIN_BLOCKS))
    step_batch_kernel(const BatchStep* __restrict__ table, int nreq, int k) {
  using T = StepTraits<R, NDIM, ISO>;
  using L = StepLayout<R, NDIM, MODE_PLAIN, ISO>;
  int lo = 0, hi = nreq - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (table[mid].cta0 <= static_cast<int>(blockIdx.x)) lo = mid;
    else hi = mid - 1;
  }
  const BatchStep& e = table[lo];
  const int n = e.n0 + k;
  if (n >= e.nlast) return;
  extern __shared__ unsigned char smem_raw[];
  StepParams* ps = reinterpret_cast<StepParams*>(smem_raw + L::SMEM);
  static_assert(sizeof(StepParams) % 4 == 0, "parameter copy by words");
  for (int i = threadIdx.x; i < static_cast<int>(sizeof(StepParams) / 4); i += blockDim.x)
    reinterpret_cast<int*>(ps)[i] = reinterpret_cast<const int*>(&e.p)[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    ps->cur = n & 1;         // level n of the request's two slots
    ps->prev = (n - 1) & 1;  // level n-1, overwritten by level n+1
  }
  if ((threadIdx.x >> 5) == T::NCW && (threadIdx.x & 31) == 0) {
    const CUtensorMap* maps[3] = {&e.maps.u, &e.maps.p, &e.maps.cm};
    for (int i = 0; i < 3; ++i)
      asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(maps[i]))
                   : "memory");
  }
  __syncthreads();
  const int local = static_cast<int>(blockIdx.x) - e.cta0;
  const int bx = local % e.tiles_x;
  const int by = (local / e.tiles_x) % e.tiles_y;
  const int z0 = local / (e.tiles_x * e.tiles_y) * ps->zchunk;
  step_body<R, NDIM, MODE_PLAIN, ISO>(e.maps.u, e.maps.p, e.maps.cm, e.maps.g, e.maps.s, *ps, bx, by, z0,
                                      min(z0 + ps->zchunk, ps->NZ));
}

}  // namespace dev

template <int R, int NDIM, bool ISO>
static cudaError_t launch_batch_iso(const BatchStep* table, int nreq, int ctas, int k, cudaStream_t stream) {
  using T = StepTraits<R, NDIM, ISO>;
  using L = StepLayout<R, NDIM, MODE_PLAIN, ISO>;
  constexpr int SMEM = L::SMEM + static_cast<int>((sizeof(StepParams) + 15) / 16 * 16);
  static_assert(SMEM <= 227 * 1024, "batched step layout exceeds the shared memory of one CTA");
  static std::atomic<unsigned long long> configured{0};
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (device & 63);
  if (!(configured.load(std::memory_order_acquire) & bit)) {
    e = cudaFuncSetAttribute(dev::step_batch_kernel<R, NDIM, ISO>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e != cudaSuccess) return e;
    configured.fetch_or(bit, std::memory_order_acq_rel);
  }
  dev::step_batch_kernel<R, NDIM, ISO><<<ctas, T::NTHREADS, SMEM, stream>>>(table, nreq, k);
  return cudaGetLastError();
}

template <int R, int NDIM>
static cudaError_t launch_batch_one(bool iso, const BatchStep* table, int nreq, int ctas, int k, cudaStream_t s) {
  if constexpr (R >= kIsoMinR) {
    if (iso) return launch_batch_iso<R, NDIM, true>(table, nreq, ctas, k, s);
  }
  return launch_batch_iso<R, NDIM, false>(table, nreq, ctas, k, s);
}

template <int R, bool ISO>
static cudaError_t launch_seg_iso(const StepMaps& maps, const StepParams& p, const SegWork& w, int ctas,
                                  cudaStream_t stream) {
  using T = StepTraits<R, 3, ISO>;
  using L = StepLayout<R, 3, MODE_PLAIN, ISO>;
  static std::atomic<unsigned long long> configured{0};
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (device & 63);
  if (!(configured.load(std::memory_order_acquire) & bit)) {
    e = cudaFuncSetAttribute(dev::step_seg_kernel<R, ISO>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
    if (e != cudaSuccess) return e;
    configured.fetch_or(bit, std::memory_order_acq_rel);
  }
  dev::step_seg_kernel<R, ISO><<<ctas, T::NTHREADS, L::SMEM, stream>>>(maps.u, maps.p, maps.cm, maps.g, maps.s, p, w);
  return cudaGetLastError();
}

template <int R>
static cudaError_t launch_seg_one(bool iso, const StepMaps& maps, const StepParams& p, const SegWork& w, int ctas,
                                  cudaStream_t s) {
  if constexpr (R >= kIsoMinR) {
    if (iso) return launch_seg_iso<R, true>(maps, p, w, ctas, s);
  }
  return launch_seg_iso<R, false>(maps, p, w, ctas, s);
}

// Host launcher for one radius; instantiated once per step_r<R>.cu.
template <int R, int NDIM, int MODE, bool ISO>
static cudaError_t launch_iso(const StepMaps& maps, const StepParams& p, dim3 grid, cudaStream_t stream) {
  using T = StepTraits<R, NDIM, ISO>;
  using L = StepLayout<R, NDIM, MODE, ISO>;
  static_assert(L::SMEM <= 227 * 1024, "step layout exceeds the shared memory of one CTA");
  static_assert(L::SMEM <= kSmemTwoCtas || L::MIN_BLOCKS == 1, "step layout does not fit its CTAs per SM");
  // the dynamic shared-memory limit is a per-device function attribute
  static std::atomic<unsigned long long> configured{0};
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (device & 63);
  if (!(configured.load(std::memory_order_acquire) & bit)) {
    e = cudaFuncSetAttribute(dev::step_kernel<R, NDIM, MODE, ISO>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
    if (e != cudaSuccess) return e;
    configured.fetch_or(bit, std::memory_order_acq_rel);
  }
  dev::step_kernel<R, NDIM, MODE, ISO><<<grid, T::NTHREADS, L::SMEM, stream>>>(maps.u, maps.p, maps.cm, maps.g, maps.s, p);
  return cudaGetLastError();
}

// p.iso selects the equal-spacing variant (instantiated from radius kIsoMinR)
template <int R, int NDIM, int MODE>
static cudaError_t launch_one(const StepMaps& maps, const StepParams& p, dim3 grid, cudaStream_t stream) {
  if constexpr (R >= kIsoMinR) {
    if (p.iso) return launch_iso<R, NDIM, MODE, true>(maps, p, grid, stream);
  }
  return launch_iso<R, NDIM, MODE, false>(maps, p, grid, stream);
}

template <int R, int NDIM>
static cudaError_t launch_modes(int mode, const StepMaps& maps, const StepParams& p, dim3 grid, cudaStream_t s) {
  switch (mode) {
    case MODE_PLAIN: return launch_one<R, NDIM, MODE_PLAIN>(maps, p, grid, s);
    case MODE_SNAP_F32: return launch_one<R, NDIM, MODE_SNAP_F32>(maps, p, grid, s);
    case MODE_SNAP_BF16: return launch_one<R, NDIM, MODE_SNAP_BF16>(maps, p, grid, s);
    case MODE_SNAP_F16: return launch_one<R, NDIM, MODE_SNAP_F16>(maps, p, grid, s);
    case MODE_GRAD_F32: return launch_one<R, NDIM, MODE_GRAD_F32>(maps, p, grid, s);
    case MODE_GRAD_BF16: return launch_one<R, NDIM, MODE_GRAD_BF16>(maps, p, grid, s);
    case MODE_GRAD_F16: return launch_one<R, NDIM, MODE_GRAD_F16>(maps, p, grid, s);
    case MODE_BORN_SRC: return launch_one<R, NDIM, MODE_BORN_SRC>(maps, p, grid, s);
    case MODE_SRC: return launch_one<R, NDIM, MODE_SRC>(maps, p, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int R, int NDIM, bool ISO>
static int smem_modes(int mode) {
  switch (mode) {
    case MODE_PLAIN: return StepLayout<R, NDIM, MODE_PLAIN, ISO>::SMEM;
    case MODE_SNAP_F32: return StepLayout<R, NDIM, MODE_SNAP_F32, ISO>::SMEM;
    case MODE_SNAP_BF16: return StepLayout<R, NDIM, MODE_SNAP_BF16, ISO>::SMEM;
    case MODE_SNAP_F16: return StepLayout<R, NDIM, MODE_SNAP_F16, ISO>::SMEM;
    case MODE_GRAD_F32: return StepLayout<R, NDIM, MODE_GRAD_F32, ISO>::SMEM;
    case MODE_GRAD_BF16: return StepLayout<R, NDIM, MODE_GRAD_BF16, ISO>::SMEM;
    case MODE_GRAD_F16: return StepLayout<R, NDIM, MODE_GRAD_F16, ISO>::SMEM;
    case MODE_BORN_SRC: return StepLayout<R, NDIM, MODE_BORN_SRC, ISO>::SMEM;
    case MODE_SRC: return StepLayout<R, NDIM, MODE_SRC, ISO>::SMEM;
    default: return -1;
  }
}

// Compile-time configuration of one step kernel, in the order documented for
// wave_step_kernel_layout; returns the number of values.
template <int R, int NDIM, int MODE, bool ISO>
static int layout_one(int* out) {
  using T = StepTraits<R, NDIM, ISO>;
  using L = StepLayout<R, NDIM, MODE, ISO>;
  const int v[] = {R, NDIM, MODE, ISO ? 1 : 0, T::BX, T::BY, T::HX, T::NTHREADS, L::MIN_BLOCKS, L::LEAD ? 1 : 0,
                   L::PF, L::NSU, L::NSP, L::QU, L::UR, L::SMEM};
  constexpr int n = sizeof(v) / sizeof(v[0]);
  for (int i = 0; i < n; ++i) out[i] = v[i];
  return n;
}

template <int R, int NDIM, bool ISO>
static int layout_modes(int mode, int* out) {
  switch (mode) {
    case MODE_PLAIN: return layout_one<R, NDIM, MODE_PLAIN, ISO>(out);
    case MODE_SNAP_F32: return layout_one<R, NDIM, MODE_SNAP_F32, ISO>(out);
    case MODE_SNAP_BF16: return layout_one<R, NDIM, MODE_SNAP_BF16, ISO>(out);
    case MODE_SNAP_F16: return layout_one<R, NDIM, MODE_SNAP_F16, ISO>(out);
    case MODE_GRAD_F32: return layout_one<R, NDIM, MODE_GRAD_F32, ISO>(out);
    case MODE_GRAD_BF16: return layout_one<R, NDIM, MODE_GRAD_BF16, ISO>(out);
    case MODE_GRAD_F16: return layout_one<R, NDIM, MODE_GRAD_F16, ISO>(out);
    case MODE_BORN_SRC: return layout_one<R, NDIM, MODE_BORN_SRC, ISO>(out);
    case MODE_SRC: return layout_one<R, NDIM, MODE_SRC, ISO>(out);
    default: return -1;
  }
}

}  // namespace wave

// Defines the per-radius entry points used by step_dispatch.cu.
#define WAVE_DEFINE_STEP_RADIUS(RR)                                                                      \
  namespace wave {                                                                                      \
  cudaError_t launch_step_r##RR(int ndim, int mode, const StepMaps& maps, const StepParams& p, dim3 grid, \
                                cudaStream_t s) {                                                       \
    return ndim == 3 ? launch_modes<RR, 3>(mode, maps, p, grid, s) : launch_modes<RR, 2>(mode, maps, p, grid, s); \
  }                                                                                                     \
  int step_smem_r##RR(int ndim, int mode, bool iso) {                                                   \
    if (iso_kernel(RR, iso))                                                                            \
      return ndim == 3 ? smem_modes<RR, 3, true>(mode) : smem_modes<RR, 2, true>(mode);                 \
    return ndim == 3 ? smem_modes<RR, 3, false>(mode) : smem_modes<RR, 2, false>(mode);                 \
  }                                                                                                     \
  cudaError_t launch_step_batch_r##RR(int ndim, bool iso, const BatchStep* table, int nreq, int ctas, int k,     \
                                      cudaStream_t s) {                                                 \
    return ndim == 3 ? launch_batch_one<RR, 3>(iso, table, nreq, ctas, k, s)                            \
                     : launch_batch_one<RR, 2>(iso, table, nreq, ctas, k, s);                           \
  }                                                                                                     \
  cudaError_t launch_step_seg_r##RR(bool iso, const StepMaps& maps, const StepParams& p, const SegWork& w, int ctas, \
                                    cudaStream_t s) {                                                   \
    return launch_seg_one<RR>(iso, maps, p, w, ctas, s);                                                \
  }                                                                                                     \
  int step_layout_r##RR(int ndim, int mode, bool iso, int* out) {                                       \
    if (iso_kernel(RR, iso))                                                                            \
      return ndim == 3 ? layout_modes<RR, 3, true>(mode, out) : layout_modes<RR, 2, true>(mode, out);   \
    return ndim == 3 ? layout_modes<RR, 3, false>(mode, out) : layout_modes<RR, 2, false>(mode, out);   \
  }                                                                                                     \
  }
