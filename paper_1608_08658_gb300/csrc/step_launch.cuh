// Host-side launch helpers of the stencil step (per radius, dimension and
// epilogue mode); included by the per-radius translation units.
#pragma once

#include <atomic>

#include "step_kernel.cuh"

namespace wave {

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
  int step_layout_r##RR(int ndim, int mode, bool iso, int* out) {                                       \
    if (iso_kernel(RR, iso))                                                                            \
      return ndim == 3 ? layout_modes<RR, 3, true>(mode, out) : layout_modes<RR, 2, true>(mode, out);   \
    return ndim == 3 ? layout_modes<RR, 3, false>(mode, out) : layout_modes<RR, 2, false>(mode, out);   \
  }                                                                                                     \
  }
