// Allocation-free objective entry point (wave_objective_noalloc).
//
// Some callers cannot allocate device memory when they need the objective:
// plug-ins embedded in a host application that owns every device allocation
// through its own pool, or services that must not touch the allocator once a
// run has started (an allocation there can stall on a device-wide
// synchronisation or fail under memory pressure at the worst moment).  For
// them this file provides one entry point that needs no workspace from the
// caller and calls no allocating routine: its per-block partial sums live in a
// file-scope device array of fixed size that every GPU loading the library
// keeps until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "wave.h"

namespace {

constexpr int kThreads = 256;
constexpr long long kChunk = WAVE_OBJECTIVE_NOALLOC_CHUNK;        // elements per block
constexpr long long kMaxN = WAVE_OBJECTIVE_NOALLOC_MAX_N;         // largest accepted n
constexpr int kMaxBlocks = static_cast<int>(kMaxN / kChunk);      // partial sums held
constexpr int kMaxDevices = 64;

// Partial sums (one per block) plus the final objective in the last slot.
static __device__ __align__(256) double g_objective_scratch[kMaxBlocks + 1];

// Residual r = d - d_obs and the FP64 sum of r^2 over one fixed chunk per
// block (fixed order inside the block: the result does not depend on timing).
__global__ void chunk_residual_kernel(const float* __restrict__ d, const float* __restrict__ dobs,
                                      float* __restrict__ r, long long n, double* __restrict__ partials) {
  __shared__ double sh[kThreads];
  const long long base = static_cast<long long>(blockIdx.x) * kChunk;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < kChunk; i += kThreads) {
    const long long k = base + i;
    if (k < n) {
      const float v = d[k] - dobs[k];
      if (r) r[k] = v;
      acc += static_cast<double>(v) * static_cast<double>(v);
    }
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void chunk_total_kernel(double* partials, int nb) {
  __shared__ double sh[kThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += kThreads) acc += partials[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[kMaxBlocks] = 0.5 * sh[0];
}

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

std::mutex g_mu;
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
// Per device: the scratch array's device address and the id of the context it
// was looked up in.  A device reset destroys that context and may reload the
// module elsewhere; the next context gets a new id, so a stale address is
// never used.
struct ScratchAddr {
  unsigned long long ctx_id = 0;
  double* addr = nullptr;
};
ScratchAddr g_scratch_addr[kMaxDevices];

// Unique id of the context current on this thread; WAVE_ERR_CUDA when there is
// none or the driver cannot report it.
int current_context_id(unsigned long long* id) {
  if (!g_ctx_current || !g_ctx_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2) {
      cudaGetLastError();
      return WAVE_ERR_CUDA;
    }
    g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    g_ctx_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext c = nullptr;
  if (g_ctx_current(&c) != CUDA_SUCCESS || !c || g_ctx_id(c, id) != CUDA_SUCCESS) return WAVE_ERR_CUDA;
  return WAVE_OK;
}

// Device address of the scratch array on `dev` (the current device).  The
// host-side symbol is only a stand-in; the address must come from the runtime,
// once per device and context.
int scratch_for(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  unsigned long long id = 0;
  if (current_context_id(&id) != WAVE_OK) return WAVE_ERR_CUDA;
  ScratchAddr& e = g_scratch_addr[dev];
  if (!e.addr || e.ctx_id != id) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_objective_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return WAVE_ERR_CUDA;
    }
    e.addr = static_cast<double*>(p);
    e.ctx_id = id;
  }
  *out = e.addr;
  return WAVE_OK;
}

bool on_device(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace

extern "C" WAVE_API int wave_objective_noalloc(const float* d, const float* d_obs, float* r_out, int64_t n,
                                               double* phi_out, void* stream) {
  if (!d || !d_obs || !phi_out || n < 0) return WAVE_ERR_INVALID_ARG;
  if (n > kMaxN) return WAVE_ERR_INVALID_ARG;
  if (n == 0) {
    *phi_out = 0.0;
    return WAVE_OK;
  }
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return WAVE_ERR_CUDA;
  }
  if (!on_device(d, dev) || !on_device(d_obs, dev) || (r_out && !on_device(r_out, dev)))
    return WAVE_ERR_INVALID_ARG;
  double* scratch = nullptr;
  int rc = scratch_for(dev, &scratch);
  if (rc != WAVE_OK) return rc;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int nb = static_cast<int>((n + kChunk - 1) / kChunk);
  chunk_residual_kernel<<<nb, kThreads, 0, s>>>(d, d_obs, r_out, n, scratch);
  chunk_total_kernel<<<1, kThreads, 0, s>>>(scratch, nb);
  if (cudaGetLastError() != cudaSuccess) return WAVE_ERR_CUDA;
  if (cudaMemcpyAsync(phi_out, scratch + kMaxBlocks, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return WAVE_ERR_CUDA;
  }
  return WAVE_OK;
}
