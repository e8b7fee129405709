// Auxiliary kernels of the wave library: model coefficients, sparse-point
// sampling and injection, residual/objective reduction, gradient fold,
// snapshot store, state packing.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ptx.cuh"
#include "wave_internal.h"

namespace wave {
namespace {

constexpr int kThreads = 256;

inline int blocks_for(long long n, int threads = kThreads, int cap = 152 * 32) {
  long long b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return static_cast<int>(b);
}

// cm = dt^2/m on the computational grid; the model inside the absorbing layer
// is the edge value of the physical model (edge replication).  Padding
// columns x >= NX are written as zero.
__global__ void setup_cm_kernel(GridDims g, const float* __restrict__ m, float* __restrict__ cm, float dt2) {
  const long long total = static_cast<long long>(g.NZ) * g.NY * g.pitch;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int x = static_cast<int>(i % g.pitch);
    const long long r = i / g.pitch;
    const int y = static_cast<int>(r % g.NY);
    const int z = static_cast<int>(r / g.NY);
    float v = 0.f;
    if (x < g.NX) {
      const int px = min(max(x - g.nblx, 0), g.PX - 1);
      const int py = min(max(y - g.nbly, 0), g.PY - 1);
      const int pz = min(max(z - g.nblz, 0), g.PZ - 1);
      v = dt2 / m[(static_cast<long long>(pz) * g.PY + py) * g.PX + px];
    }
    cm[i] = v;
  }
}

// A physical field extended onto the computational grid by edge replication
// (the padding of the model, applied to a model perturbation).
__global__ void pad_field_kernel(GridDims g, const float* __restrict__ phys, float* __restrict__ comp) {
  const long long total = static_cast<long long>(g.NZ) * g.NY * g.pitch;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int x = static_cast<int>(i % g.pitch);
    const long long r = i / g.pitch;
    const int y = static_cast<int>(r % g.NY);
    const int z = static_cast<int>(r / g.NY);
    float v = 0.f;
    if (x < g.NX) {
      const int px = min(max(x - g.nblx, 0), g.PX - 1);
      const int py = min(max(y - g.nbly, 0), g.PY - 1);
      const int pz = min(max(z - g.nblz, 0), g.PZ - 1);
      v = phys[(static_cast<long long>(pz) * g.PY + py) * g.PX + px];
    }
    comp[i] = v;
  }
}

// min and max of a positive float array via the ordering of IEEE bit patterns.
__global__ void minmax_kernel(const float* __restrict__ m, long long n, unsigned int* out) {
  unsigned int lo = 0xffffffffu, hi = 0u;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const unsigned int b = __float_as_uint(m[i]);
    // non-positive values and NaN map to extreme keys so that the host rejects them
    const unsigned int key = (b >> 31) ? 0u : b;
    lo = min(lo, key);
    hi = max(hi, key);
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, off));
    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(out, lo);
    atomicMax(out + 1, hi);
  }
}

// Receiver sampling: one group of 2^ndim lanes per point, each lane one
// corner; the group sums its weighted corners with xor shuffles.
__global__ void gather_kernel(GatherSet gs, const float* __restrict__ field, float* __restrict__ out) {
  const int C = gs.ndim == 3 ? 8 : 4;
  const long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  const long long pt = t / C;
  const int c = static_cast<int>(t % C);
  const bool valid = pt < gs.n;
  float v = 0.f;
  if (valid) {
    const float fx = gs.frac[3 * pt], fy = gs.frac[3 * pt + 1], fz = gs.frac[3 * pt + 2];
    const int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
    float w = (bx ? fx : 1.f - fx) * (by ? fy : 1.f - fy);
    if (gs.ndim == 3) w *= (bz ? fz : 1.f - fz);
    const long long idx = gs.base[pt] + bx + by * gs.sy + bz * gs.sz;
    v = __fmul_rn(w, field[idx]);  // never fused with the reduction below
  }
  for (int off = C / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if (valid && c == 0) out[pt] = v;
}

__device__ __forceinline__ void decode_cell(long long cell, const GridDims& g, int& x, int& y, int& z) {
  x = static_cast<int>(cell % g.pitch);
  const long long r = cell / g.pitch;
  y = static_cast<int>(r % g.NY);
  z = static_cast<int>(r / g.NY);
}

// Per injected cell: cm/(1+k) with the same damping expression as the step.
__global__ void inject_coef_kernel(InjectSet is, GridDims g, const float* __restrict__ cm, float emx, float emy,
                                   float emz, float half_inv_dt) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= is.n) return;
  const long long cell = is.cell[k];
  int x, y, z;
  decode_cell(cell, g, x, y, z);
  // the same operations, in the same order, as the step kernel's damping
  float eta = dev::sponge_sum(dev::sponge_term(x, g.NX, g.nblx, emx), dev::sponge_term(y, g.NY, g.nbly, emy));
  if (g.NZ > 1) eta = dev::sponge_sum(eta, dev::sponge_term(z, g.NZ, g.nblz, emz));
  const float c = cm[cell];
  const float kk = __fmul_rn(__fmul_rn(eta, c), half_inv_dt);
  const float inv = eta == 0.f ? 1.f : __fdividef(1.f, __fadd_rn(1.f, kk));
  is.coef[k] = c * inv;
}

// Injection of P^T values into the new level, one thread per unique cell
// (entries of a cell summed in a fixed order: no atomics, deterministic).
__global__ void inject_kernel(InjectSet is, const float* __restrict__ vals, float* __restrict__ field) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= is.n) return;
  float s = 0.f;
  for (int e = is.rowptr[k]; e < is.rowptr[k + 1]; ++e) s = fmaf(is.w[e], vals[is.pidx[e]], s);
  field[is.cell[k]] = fmaf(is.coef[k], s, field[is.cell[k]]);
}

__device__ __forceinline__ float snap_value(const void* snap, int fmt, const float* scale, long long cell,
                                            const GridDims& g, int slabs_x, int slabs_y) {
  if (fmt == 0) return static_cast<const float*>(snap)[cell];
  int x, y, z;
  decode_cell(cell, g, x, y, z);
  const float s = scale[(static_cast<long long>(z) * slabs_y + (y >> 1)) * slabs_x + (x >> 6)];
  const uint16_t h = static_cast<const uint16_t*>(snap)[cell];
  float v;
  if (fmt == 1) {
    __nv_bfloat16_raw r;
    r.x = h;
    v = __bfloat162float(__nv_bfloat16(r));
  } else {
    __half_raw r;
    r.x = h;
    v = __half2float(__half(r));
  }
  return v * s;
}

// Injection during the gradient sweep: the step kernel formed the imaging
// term with the new level before injection; add the missing part
// -u^j * delta / dt^2 at the injected cells.
__global__ void inject_grad_kernel(InjectSet is, const float* __restrict__ vals, float* __restrict__ field,
                                   float* __restrict__ grad, const void* snap, int fmt, const float* scale, GridDims g,
                                   int slabs_x, int slabs_y, float inv_dt2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= is.n) return;
  float s = 0.f;
  for (int e = is.rowptr[k]; e < is.rowptr[k + 1]; ++e) s = fmaf(is.w[e], vals[is.pidx[e]], s);
  const long long cell = is.cell[k];
  const float delta = is.coef[k] * s;
  field[cell] += delta;
  grad[cell] -= snap_value(snap, fmt, scale, cell, g, slabs_x, slabs_y) * delta * inv_dt2;
}

// r = d - d_obs and per-block partial sums of r^2 in FP64 (fixed tree order).
__global__ void residual_kernel(const float* __restrict__ d, const float* __restrict__ dobs, float* __restrict__ r,
                                long long n, double* __restrict__ partials) {
  __shared__ double sh[kThreads];
  double acc = 0.0;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const float v = d[i] - dobs[i];
    r[i] = v;
    acc += static_cast<double>(v) * static_cast<double>(v);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void sum_partials_kernel(const double* __restrict__ partials, int n, double* out) {
  __shared__ double sh[kThreads];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partials[i];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = 0.5 * sh[0];
}

// Transpose of the edge-replicating padding: each physical cell sums the
// computational cells that were copied from it.
__global__ void fold_kernel(GridDims g, const float* __restrict__ gc, float* __restrict__ gp) {
  const long long total = static_cast<long long>(g.PZ) * g.PY * g.PX;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int px = static_cast<int>(i % g.PX);
    const long long r = i / g.PX;
    const int py = static_cast<int>(r % g.PY);
    const int pz = static_cast<int>(r / g.PY);
    const int xlo = px == 0 ? 0 : px + g.nblx, xhi = px == g.PX - 1 ? g.NX - 1 : px + g.nblx;
    const int ylo = py == 0 ? 0 : py + g.nbly, yhi = py == g.PY - 1 ? g.NY - 1 : py + g.nbly;
    const int zlo = pz == 0 ? 0 : pz + g.nblz, zhi = pz == g.PZ - 1 ? g.NZ - 1 : pz + g.nblz;
    float acc = 0.f;
    for (int z = zlo; z <= zhi; ++z)
      for (int y = ylo; y <= yhi; ++y) {
        const float* row = gc + (static_cast<long long>(z) * g.NY + y) * g.pitch;
        for (int x = xlo; x <= xhi; ++x) acc += row[x];
      }
    gp[i] = acc;
  }
}

// Store one wavefield level as a snapshot: one warp per 64 x 2 slab, the
// same lane layout and scale rule as the fused store of the step kernel.
__global__ void snapshot_store_kernel(GridDims g, const float* __restrict__ field, void* snap, float* scale, int fmt,
                                      int slabs_x, int slabs_y) {
  const int warp_global = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const long long nslabs = static_cast<long long>(slabs_x) * slabs_y * g.NZ;
  if (warp_global >= nslabs) return;
  const int lane = threadIdx.x & 31;
  const int sx = static_cast<int>(warp_global % slabs_x);
  const long long r = warp_global / slabs_x;
  const int sy = static_cast<int>(r % slabs_y);
  const int z = static_cast<int>(r / slabs_y);
  const int x = sx * kSlabX + 4 * (lane & 15);
  const int y = sy * kSlabY + (lane >> 4);
  const bool ok = x < g.NX && y < g.NY;
  const long long idx = (static_cast<long long>(z) * g.NY + y) * g.pitch + x;
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (ok) v = *reinterpret_cast<const float4*>(field + idx);
  if (fmt == 0) {
    if (ok) *reinterpret_cast<float4*>(static_cast<float*>(snap) + idx) = v;
    return;
  }
  const float lmax = fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)));
  const float amax = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(lmax)));
  const float s = dev::slab_scale(amax);
  const float is = dev::slab_inv_scale(s);
  if (ok) {
    uint2 u;
    if (fmt == 1) {
      __nv_bfloat162 a = __floats2bfloat162_rn(v.x * is, v.y * is);
      __nv_bfloat162 b = __floats2bfloat162_rn(v.z * is, v.w * is);
      u.x = *reinterpret_cast<uint32_t*>(&a);
      u.y = *reinterpret_cast<uint32_t*>(&b);
    } else {
      __half2 a = __floats2half2_rn(v.x * is, v.y * is);
      __half2 b = __floats2half2_rn(v.z * is, v.w * is);
      u.x = *reinterpret_cast<uint32_t*>(&a);
      u.y = *reinterpret_cast<uint32_t*>(&b);
    }
    *reinterpret_cast<uint2*>(static_cast<uint16_t*>(snap) + idx) = u;
  }
  if (lane == 0) scale[(static_cast<long long>(z) * slabs_y + sy) * slabs_x + sx] = s;
}

__global__ void pack_kernel(GridDims g, const float* __restrict__ field, float* __restrict__ dense) {
  const long long total = static_cast<long long>(g.NZ) * g.NY * g.NX;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int x = static_cast<int>(i % g.NX);
    const long long r = i / g.NX;
    dense[i] = field[r * g.pitch + x];
  }
}

__global__ void unpack_kernel(GridDims g, const float* __restrict__ dense, float* __restrict__ field) {
  const long long total = static_cast<long long>(g.NZ) * g.NY * g.NX;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < total;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    const int x = static_cast<int>(i % g.NX);
    const long long r = i / g.NX;
    field[r * g.pitch + x] = dense[i];
  }
}

// Variants used inside captured CUDA graphs: the time row is read from a
// device counter (the number of steps completed before the replay) plus the
// position of the step within the captured chunk.
__global__ void inject_counter_kernel(InjectSet is, const float* __restrict__ q, long long ns,
                                      const int* __restrict__ counter, int offset, float* __restrict__ field) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= is.n) return;
  const float* vals = q + static_cast<long long>(*counter + offset) * ns;
  float s = 0.f;
  for (int e = is.rowptr[k]; e < is.rowptr[k + 1]; ++e) s = fmaf(is.w[e], vals[is.pidx[e]], s);
  field[is.cell[k]] = fmaf(is.coef[k], s, field[is.cell[k]]);
}

__global__ void gather_counter_kernel(GatherSet gs, const float* __restrict__ field, float* __restrict__ d,
                                      const int* __restrict__ counter, int offset) {
  const int C = gs.ndim == 3 ? 8 : 4;
  const long long t = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
  const long long pt = t / C;
  const int c = static_cast<int>(t % C);
  const bool valid = pt < gs.n;
  float v = 0.f;
  if (valid) {
    const float fx = gs.frac[3 * pt], fy = gs.frac[3 * pt + 1], fz = gs.frac[3 * pt + 2];
    const int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
    float w = (bx ? fx : 1.f - fx) * (by ? fy : 1.f - fy);
    if (gs.ndim == 3) w *= (bz ? fz : 1.f - fz);
    v = __fmul_rn(w, field[gs.base[pt] + bx + by * gs.sy + bz * gs.sz]);
  }
  for (int off = C / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if (valid && c == 0) d[static_cast<long long>(*counter + offset) * gs.n + pt] = v;
}

// Batched injection of the serving path: CTA r injects row n = n0 + k of
// request r into its level n+1 (the arithmetic of inject_kernel).
__global__ void inject_batch_kernel(const BatchSparse* __restrict__ table, int k) {
  const BatchSparse& e = table[blockIdx.x];
  const int n = e.n0 + k;
  if (n >= e.nlast || e.inj.n == 0) return;
  const float* vals = e.q + static_cast<long long>(n) * e.ns;
  float* field = e.fields + ((n + 1) & 1) * e.slot_elems;
  for (int c = threadIdx.x; c < e.inj.n; c += blockDim.x) {
    float s = 0.f;
    for (int i = e.inj.rowptr[c]; i < e.inj.rowptr[c + 1]; ++i) s = fmaf(e.inj.w[i], vals[e.inj.pidx[i]], s);
    field[e.inj.cell[c]] = fmaf(e.inj.coef[c], s, field[e.inj.cell[c]]);
  }
}

// Batched receiver sampling: the gather CTAs of the requests follow one
// another (first CTA gcta0); CTA j of request r samples row n + 1 from its
// level n+1 with the lane layout and reduction of gather_kernel.
__global__ void gather_batch_kernel(const BatchSparse* __restrict__ table, int nreq, int k) {
  int lo = 0, hi = nreq - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (table[mid].gcta0 <= static_cast<int>(blockIdx.x)) lo = mid;
    else hi = mid - 1;
  }
  const BatchSparse& e = table[lo];
  const int n = e.n0 + k;
  const GatherSet& gs = e.gat;
  if (n >= e.nlast || gs.n == 0) return;
  const float* field = e.fields + ((n + 1) & 1) * e.slot_elems;
  const int C = gs.ndim == 3 ? 8 : 4;
  const long long t = (static_cast<long long>(blockIdx.x) - e.gcta0) * blockDim.x + threadIdx.x;
  const long long pt = t / C;
  const int c = static_cast<int>(t % C);
  const bool valid = pt < gs.n;
  float v = 0.f;
  if (valid) {
    const float fx = gs.frac[3 * pt], fy = gs.frac[3 * pt + 1], fz = gs.frac[3 * pt + 2];
    const int bx = c & 1, by = (c >> 1) & 1, bz = (c >> 2) & 1;
    float w = (bx ? fx : 1.f - fx) * (by ? fy : 1.f - fy);
    if (gs.ndim == 3) w *= (bz ? fz : 1.f - fz);
    v = __fmul_rn(w, field[gs.base[pt] + bx + by * gs.sy + bz * gs.sz]);
  }
  for (int off = C / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if (valid && c == 0) e.d[static_cast<long long>(n + 1) * gs.n + pt] = v;
}

__global__ void counter_add_kernel(int* counter, int delta) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *counter += delta;
}

__global__ void fill_zero_kernel(float* p, long long n) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    p[i] = 0.f;
}

}  // namespace

cudaError_t launch_setup_cm(const GridDims& g, const float* m_phys, float* cm, float dt2, cudaStream_t s) {
  const long long n = static_cast<long long>(g.NZ) * g.NY * g.pitch;
  setup_cm_kernel<<<blocks_for(n), kThreads, 0, s>>>(g, m_phys, cm, dt2);
  return cudaGetLastError();
}

cudaError_t launch_pad_field(const GridDims& g, const float* phys, float* comp, cudaStream_t s) {
  const long long n = static_cast<long long>(g.NZ) * g.NY * g.pitch;
  pad_field_kernel<<<blocks_for(n), kThreads, 0, s>>>(g, phys, comp);
  return cudaGetLastError();
}

cudaError_t launch_minmax(const float* m, long long n, unsigned int* out, cudaStream_t s) {
  minmax_kernel<<<blocks_for(n), kThreads, 0, s>>>(m, n, out);
  return cudaGetLastError();
}

cudaError_t launch_gather(const GatherSet& gs, const float* field, float* out_row, cudaStream_t s) {
  if (gs.n == 0) return cudaSuccess;
  const long long lanes = gs.n * (gs.ndim == 3 ? 8 : 4);
  const long long blocks = (lanes + kThreads - 1) / kThreads;
  gather_kernel<<<static_cast<unsigned>(blocks), kThreads, 0, s>>>(gs, field, out_row);
  return cudaGetLastError();
}

cudaError_t launch_inject_coef(const InjectSet& is, const GridDims& g, const float* cm, const float* em,
                               float half_inv_dt, cudaStream_t s) {
  if (is.n == 0) return cudaSuccess;
  inject_coef_kernel<<<(is.n + kThreads - 1) / kThreads, kThreads, 0, s>>>(is, g, cm, em[0], em[1], em[2],
                                                                            half_inv_dt);
  return cudaGetLastError();
}

cudaError_t launch_inject(const InjectSet& is, const float* values_row, float* field, cudaStream_t s) {
  if (is.n == 0) return cudaSuccess;
  inject_kernel<<<(is.n + kThreads - 1) / kThreads, kThreads, 0, s>>>(is, values_row, field);
  return cudaGetLastError();
}

cudaError_t launch_inject_grad(const InjectSet& is, const float* values_row, float* field, float* grad,
                               const void* snap_level, int snap_fmt, const float* scale_level, const GridDims& g,
                               int slabs_x, int slabs_y, float inv_dt2, cudaStream_t s) {
  if (is.n == 0) return cudaSuccess;
  inject_grad_kernel<<<(is.n + kThreads - 1) / kThreads, kThreads, 0, s>>>(
      is, values_row, field, grad, snap_level, snap_fmt, scale_level, g, slabs_x, slabs_y, inv_dt2);
  return cudaGetLastError();
}

int residual_blocks(long long n) { return blocks_for(n, kThreads, 1024); }

int gather_batch_ctas(long long npoints, int ndim) {
  const long long lanes = npoints * (ndim == 3 ? 8 : 4);
  return static_cast<int>((lanes + kThreads - 1) / kThreads);
}

cudaError_t launch_inject_batch(const BatchSparse* table, int nreq, int k, cudaStream_t s) {
  if (nreq <= 0) return cudaSuccess;
  inject_batch_kernel<<<nreq, 64, 0, s>>>(table, k);
  return cudaGetLastError();
}

cudaError_t launch_gather_batch(const BatchSparse* table, int nreq, int gather_ctas, int k, cudaStream_t s) {
  if (nreq <= 0 || gather_ctas <= 0) return cudaSuccess;
  gather_batch_kernel<<<gather_ctas, kThreads, 0, s>>>(table, nreq, k);
  return cudaGetLastError();
}

cudaError_t launch_residual(const float* d, const float* d_obs, float* r, long long n, double* partials,
                            int nblocks, cudaStream_t s) {
  residual_kernel<<<nblocks, kThreads, 0, s>>>(d, d_obs, r, n, partials);
  return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double* partials, int n, double* out, cudaStream_t s) {
  sum_partials_kernel<<<1, kThreads, 0, s>>>(partials, n, out);
  return cudaGetLastError();
}

cudaError_t launch_fold(const GridDims& g, const float* grad_comp, float* grad_phys, cudaStream_t s) {
  const long long n = static_cast<long long>(g.PZ) * g.PY * g.PX;
  fold_kernel<<<blocks_for(n), kThreads, 0, s>>>(g, grad_comp, grad_phys);
  return cudaGetLastError();
}

cudaError_t launch_snapshot_store(const GridDims& g, const float* field, void* snap, float* scale, int fmt,
                                  int slabs_x, int slabs_y, cudaStream_t s) {
  const long long nslabs = static_cast<long long>(slabs_x) * slabs_y * g.NZ;
  const long long blocks = (nslabs + 7) / 8;
  snapshot_store_kernel<<<static_cast<unsigned>(blocks), kThreads, 0, s>>>(g, field, snap, scale, fmt, slabs_x,
                                                                           slabs_y);
  return cudaGetLastError();
}

cudaError_t launch_pack_state(const GridDims& g, const float* field, float* dense, cudaStream_t s) {
  const long long n = static_cast<long long>(g.NZ) * g.NY * g.NX;
  pack_kernel<<<blocks_for(n), kThreads, 0, s>>>(g, field, dense);
  return cudaGetLastError();
}

cudaError_t launch_unpack_state(const GridDims& g, const float* dense, float* field, cudaStream_t s) {
  const long long n = static_cast<long long>(g.NZ) * g.NY * g.NX;
  unpack_kernel<<<blocks_for(n), kThreads, 0, s>>>(g, dense, field);
  return cudaGetLastError();
}

cudaError_t launch_inject_counter(const InjectSet& is, const float* q, long long ns, const int* counter, int offset,
                                  float* field, cudaStream_t s) {
  if (is.n == 0) return cudaSuccess;
  inject_counter_kernel<<<(is.n + kThreads - 1) / kThreads, kThreads, 0, s>>>(is, q, ns, counter, offset, field);
  return cudaGetLastError();
}

cudaError_t launch_gather_counter(const GatherSet& gs, const float* field, float* d, const int* counter, int offset,
                                  cudaStream_t s) {
  if (gs.n == 0) return cudaSuccess;
  const long long lanes = gs.n * (gs.ndim == 3 ? 8 : 4);
  const long long blocks = (lanes + kThreads - 1) / kThreads;
  gather_counter_kernel<<<static_cast<unsigned>(blocks), kThreads, 0, s>>>(gs, field, d, counter, offset);
  return cudaGetLastError();
}

cudaError_t launch_counter_add(int* counter, int delta, cudaStream_t s) {
  counter_add_kernel<<<1, 32, 0, s>>>(counter, delta);
  return cudaGetLastError();
}

cudaError_t launch_fill_zero(float* p, long long n, cudaStream_t s) {
  fill_zero_kernel<<<blocks_for(n), kThreads, 0, s>>>(p, n);
  return cudaGetLastError();
}

}  // namespace wave
