// One leapfrog time level of the damped acoustic operator (Listing 1 / Eq. 1),
// which is also one level of its adjoint (Listing 2): with
//   a = m/dt^2 + eta/(2dt), b = 2m/dt^2 + L, c = m/dt^2 - eta/(2dt)
// the new level is (b*cur - c*prev)/a; dividing by m/dt^2 and writing
// cm = dt^2/m, k = eta*cm/(2dt):
//   new = (2*cur - (1-k)*prev + cm*L(cur)) / (1+k).
// The adjoint recursion lam_{j-1} = (b lam_j - c lam_{j+1} + ...)/a has the
// same form, so one kernel serves both; the epilogue variant adds a snapshot
// store (forward with storage for Eq. 3) or the imaging condition of Eq. 3
//   g -= u^j * (lam_{j-1} - 2 lam_j + lam_{j+1}) / dt^2 .
//
// Data movement (3D): a CTA owns a BX x BY column tile and streams a chunk of
// planes along axis 2.  A producer warp issues TMA tile loads into two rings
// of mbarrier-tracked stages: the queue-feed ring (halo planes of the centre
// level in the classic layout; interior boxes of plane z+R in the lead-plane
// layout) and the per-point ring (previous level, cm, and g / snapshot / dm /
// S by mode; plus the centre halo box in the lead-plane layout).  BY/2
// consumer warps keep the 2R+1 centre-level values of their columns in a
// register queue (the z taps), read x/y taps from shared memory, and write the
// new level with 16-byte stores.  The layout, prefetch depth, plane grouping
// and occupancy of each (R, NDIM, MODE, ISO) are set by StepLayout.
// Zero ghost values outside the grid come from the TMA out-of-bounds fill.
// Every barrier wait is bounded; on expiry the kernel records a timeout in the
// status word, drains its own copies and returns.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "ptx.cuh"
#include "wave_internal.h"

namespace wave {
namespace dev {

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }

// 1/(1+k) and 1-k of the damped update.  1+k >= 1 is a moderate number, for
// which the fast division intrinsic is within 2 ulp; the correctly rounded
// reciprocal costs a longer instruction sequence at every sponge point.  The
// source-injection coefficient uses the same expression.
__device__ __forceinline__ float damp_inv(float eta, float cm, float half_inv_dt, float& one_minus_k) {
  const float k = __fmul_rn(__fmul_rn(eta, cm), half_inv_dt);
  one_minus_k = __fsub_rn(1.f, k);
  return eta == 0.f ? 1.f : __fdividef(1.f, __fadd_rn(1.f, k));
}

template <int FMT>
__device__ __forceinline__ void store_snap4(void* base, long long idx, const float4& v, float inv_s) {
  if (FMT == 0) {
    *reinterpret_cast<float4*>(static_cast<float*>(base) + idx) = v;
  } else if (FMT == 1) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v.x * inv_s, v.y * inv_s);
    __nv_bfloat162 b = __floats2bfloat162_rn(v.z * inv_s, v.w * inv_s);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t*>(&a);
    u.y = *reinterpret_cast<uint32_t*>(&b);
    *reinterpret_cast<uint2*>(static_cast<uint16_t*>(base) + idx) = u;
  } else {
    __half2 a = __floats2half2_rn(v.x * inv_s, v.y * inv_s);
    __half2 b = __floats2half2_rn(v.z * inv_s, v.w * inv_s);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t*>(&a);
    u.y = *reinterpret_cast<uint32_t*>(&b);
    *reinterpret_cast<uint2*>(static_cast<uint16_t*>(base) + idx) = u;
  }
}

template <int FMT>
__device__ __forceinline__ float4 load_snap4_smem(const unsigned char* p, float s) {
  if (FMT == 0) return *reinterpret_cast<const float4*>(p);
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  float2 a, b;
  if (FMT == 1) {
    a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
    b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
  } else {
    a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
    b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
  }
  return make_float4(a.x * s, a.y * s, b.x * s, b.y * s);
}

// compile-time plane offset inside a group of planes
template <int V>
struct IntC {
  static constexpr int value = V;
};

// Calls f(IntC<0>{}), f(IntC<1>{}), ... in order while they return true.
template <typename F, int I, int N>
__device__ __forceinline__ bool call_in_order(F& f, IntC<I>, IntC<N>) {
  if constexpr (I == N) {
    return true;
  } else {
    if (!f(IntC<I>{})) return false;
    return call_in_order(f, IntC<I + 1>{}, IntC<N>{});
  }
}

// Producer warp of a step kernel (layout L: StepLayout or Step2Layout).  Lane
// 0 streams the CTA's planes through the two rings: the queue-feed stage of
// sequence s (the centre-level halo plane z0 - RZ + s, or in the lead-plane
// layout its interior box) and, from s = 2 RZ on, the per-point stage of plane
// j = s - 2 RZ (previous level, cm, and g / snapshot by mode; plus the centre
// halo box in the lead-plane layout).  A stage is refilled once the consumer
// warps have released it.  When a wait runs out, or the consumers abort, the
// producer records the timeout and lets every copy it issued land.
template <class L, int R, int MODE>
__device__ __forceinline__ void produce(const CUtensorMap& tm_u, const CUtensorMap& tm_p, const CUtensorMap& tm_cm,
                                        const CUtensorMap& tm_g, const CUtensorMap& tm_s, const StepParams& p,
                                        int x0, int y0, int z0, int nU, uint64_t* fullU, uint64_t* emptyU,
                                        uint64_t* fullP, uint64_t* emptyP, volatile int* abort_flag, float* Ubase,
                                        unsigned char* Pbase) {
  constexpr int RZ = L::RZ;
  const int lane = threadIdx.x & 31;
  // failure-detection test hook: with no load issued, the consumers' waits
  // run out after p.wait_ns and take the timeout path; nothing is in flight
  if (p.withhold) return;
  if (lane != 0) return;
  prefetch_tensormap(&tm_u);
  prefetch_tensormap(&tm_p);
  prefetch_tensormap(&tm_cm);
  if (mode_loads_g(MODE)) prefetch_tensormap(&tm_g);
  if (mode_is_grad(MODE)) prefetch_tensormap(&tm_s);
  bool ok = true;
  if constexpr (L::COMBINED) {
    // one ring: stage s = queue box of plane z0 - RZ + S0 + s plus, from
    // s = 2RZ - S0 on, the per-point tiles of plane s + S0 - 2RZ, under
    // fullU/emptyU[s % NSU]; S0 = 2RZ where the consumers load the first 2RZ
    // queue planes themselves (L::DIRECT_FILL), else 0
    constexpr int NS = L::NSU;
    constexpr int S0 = L::DIRECT_FILL ? 2 * RZ : 0;
    static_assert(L::NSU == L::NSP, "one stage per plane for both rings");
    int issued = 0;
    for (int s = 0; s < nU; ++s) {
      const int slot = s % NS;
      if (s >= NS) ok = mbar_wait_bounded(&emptyU[slot], ((s / NS) - 1) & 1, abort_flag, p.wait_ns);
      if (!ok) break;
      const bool tiles = s + S0 >= 2 * RZ;
      mbar_arrive_expect_tx(&fullU[slot], L::Q_BYTES + (tiles ? L::P_TX : 0));
      tma_load_4d(Ubase + slot * (L::Q_STRIDE / 4), &tm_p, x0, y0, z0 - RZ + S0 + s, p.cur, &fullU[slot]);
      if (tiles) {
        const int j = s + S0 - 2 * RZ;
        unsigned char* pd = Pbase + slot * L::P_BYTES;
        tma_load_4d(pd + L::HALO_OFF, &tm_u, x0 - L::HX, y0 - R, z0 + j, p.cur, &fullU[slot]);
        tma_load_4d(pd + L::PREV_OFF, &tm_p, x0, y0, z0 + j, p.prev, &fullU[slot]);
        tma_load_3d(pd + L::CM_OFF, &tm_cm, x0, y0, z0 + j, &fullU[slot]);
        if (mode_loads_g(MODE)) tma_load_3d(pd + L::G_OFF, &tm_g, x0, y0, z0 + j, &fullU[slot]);
        if (mode_is_grad(MODE)) tma_load_4d(pd + L::S_OFF, &tm_s, x0, y0, z0 + j, p.snap_level, &fullU[slot]);
      }
      issued = s + 1;
    }
    if (!ok) {
      *abort_flag = 1;
      atomicExch(p.status, kDevTimeout);
    }
    if (*abort_flag) {
      for (int slot = 0; slot < NS; ++slot) {
        if (issued > slot) {
          const int last = slot + NS * ((issued - 1 - slot) / NS);
          mbar_wait_bounded(&fullU[slot], (last / NS) & 1, nullptr, kWaitLimitNs);
        }
      }
    }
    return;
  }
  int issuedU = 0, issuedP = 0;
  for (int s = 0; s < nU; ++s) {
    const int slot = s % L::NSU;
    if (s >= L::NSU) ok = mbar_wait_bounded(&emptyU[slot], ((s / L::NSU) - 1) & 1, abort_flag, p.wait_ns);
    if (!ok) break;
    mbar_arrive_expect_tx(&fullU[slot], L::Q_BYTES);
    if constexpr (L::LEAD)
      tma_load_4d(Ubase + slot * (L::Q_STRIDE / 4), &tm_p, x0, y0, z0 - RZ + s, p.cur, &fullU[slot]);
    else
      tma_load_4d(Ubase + slot * (L::Q_STRIDE / 4), &tm_u, x0 - L::HX, y0 - R, z0 - RZ + s, p.cur, &fullU[slot]);
    issuedU = s + 1;
    if (s >= 2 * RZ) {
      const int j = s - 2 * RZ;
      const int ps = j % L::NSP;
      if (j >= L::NSP) ok = mbar_wait_bounded(&emptyP[ps], ((j / L::NSP) - 1) & 1, abort_flag, p.wait_ns);
      if (!ok) break;
      unsigned char* pd = Pbase + ps * L::P_BYTES;
      mbar_arrive_expect_tx(&fullP[ps], L::P_TX);
      if constexpr (L::LEAD)
        tma_load_4d(pd + L::HALO_OFF, &tm_u, x0 - L::HX, y0 - R, z0 + j, p.cur, &fullP[ps]);
      tma_load_4d(pd + L::PREV_OFF, &tm_p, x0, y0, z0 + j, p.prev, &fullP[ps]);
      tma_load_3d(pd + L::CM_OFF, &tm_cm, x0, y0, z0 + j, &fullP[ps]);
      if (mode_loads_g(MODE)) tma_load_3d(pd + L::G_OFF, &tm_g, x0, y0, z0 + j, &fullP[ps]);
      if (mode_is_grad(MODE)) tma_load_4d(pd + L::S_OFF, &tm_s, x0, y0, z0 + j, p.snap_level, &fullP[ps]);
      issuedP = j + 1;
    }
  }
  if (!ok) {
    *abort_flag = 1;
    atomicExch(p.status, kDevTimeout);
  }
  if (*abort_flag) {
    // let every copy this thread issued land before the CTA exits
    for (int slot = 0; slot < L::NSU; ++slot) {
      if (issuedU > slot) {
        const int last = slot + L::NSU * ((issuedU - 1 - slot) / L::NSU);
        mbar_wait_bounded(&fullU[slot], (last / L::NSU) & 1, nullptr, kWaitLimitNs);
      }
    }
    for (int slot = 0; slot < L::NSP; ++slot) {
      if (issuedP > slot) {
        const int last = slot + L::NSP * ((issuedP - 1 - slot) / L::NSP);
        mbar_wait_bounded(&fullP[slot], (last / L::NSP) & 1, nullptr, kWaitLimitNs);
      }
    }
  }
}

// No extra work for the consumer warps before the first plane.
struct NoPre {
  __device__ __forceinline__ void operator()(int) const {}
};

// Body of one step for the CTA at tile (bx, by), output planes z0 .. z1-1 of
// its column; the step kernel below runs it once per CTA, the batched step of
// the serving path for the CTAs of several requests, the segmented step once
// per column segment of the CTA.  `pre(consumer thread index)` runs on the
// consumer warps while the producer issues the first loads.
template <int R, int NDIM, int MODE, bool ISO, class Pre = NoPre>
__device__ __forceinline__ void step_body(const CUtensorMap& tm_u, const CUtensorMap& tm_p, const CUtensorMap& tm_cm,
                                          const CUtensorMap& tm_g, const CUtensorMap& tm_s, const StepParams& p,
                                          int bx, int by, int z0, int z1, Pre&& pre = Pre{}) {
  using T = StepTraits<R, NDIM, ISO>;
  using L = StepLayout<R, NDIM, MODE, ISO>;
  constexpr int RZ = T::RZ;
  constexpr int FMT = mode_snap_fmt(MODE);

  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  uint64_t* fullU = reinterpret_cast<uint64_t*>(smem);
  uint64_t* emptyU = fullU + L::NSU;
  uint64_t* fullP = emptyU + L::NSU;
  uint64_t* emptyP = fullP + L::NSP;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(emptyP + L::NSP);
  float* Ubase = reinterpret_cast<float*>(smem + L::U_OFF);
  unsigned char* Pbase = smem + L::PST_OFF;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int x0 = bx * T::BX;
  const int y0 = by * T::BY;
  const int nP = z1 - z0;
  const int nU = nP + (L::DIRECT_FILL ? 0 : 2 * RZ);  // stages the producer streams
  if (nP <= 0) return;

  if (tid == 0) {
    for (int i = 0; i < L::NSU; ++i) {
      mbar_init(&fullU[i], 1);
      mbar_init(&emptyU[i], T::NCW);
    }
    for (int i = 0; i < L::NSP; ++i) {
      mbar_init(&fullP[i], 1);
      mbar_init(&emptyP[i], T::NCW);
    }
    *abort_flag = 0;
    fence_mbarrier_init();
  }
  __syncthreads();

  // ------------------------------------------------------------------ producer
  if (warp == T::NCW) {
    produce<L, R, MODE>(tm_u, tm_p, tm_cm, tm_g, tm_s, p, x0, y0, z0, nU, fullU, emptyU, fullP, emptyP,
                        abort_flag, Ubase, Pbase);
    return;
  }

  // ------------------------------------------------------------------ consumers
  pre(tid);
  const int ty = tid >> 4;  // row of the tile, 0..BY-1
  const int tx = tid & 15;  // quad of 4 x points
  const int gx = x0 + 4 * tx;
  const int gy = y0 + ty;
  const bool store_ok = (gx < p.NX) && (gy < p.NY);
  const int lofs = (R + ty) * T::UW + T::HX + 4 * tx;  // centre of this quad in a halo box
  const int tofs = (ty * T::BX + 4 * tx) * 4;          // byte offset of this quad in a tile
  const int qofs = L::LEAD ? tofs / 4 : lofs;           // this quad in a queue-feed stage

  // sponge along x (per point) and axis 1 (per row)
  const float ey = sponge_term(gy, p.NY, p.nbly, p.emy);
  float exy[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) exy[i] = sponge_sum(sponge_term(gx + i, p.NX, p.nblx, p.emx), ey);
  // all terms are >= 0: the column is undamped iff the largest is zero
  const float exy_max = fmaxf(fmaxf(exy[0], exy[1]), fmaxf(exy[2], exy[3]));

  // Coefficients as packed pairs (loop invariant).  With different spacings
  // per axis there are 3R of them, which up to radius 6 fit in registers;
  // above, the multiply takes the scalar coefficient from the parameter bank
  // and only the sums stay packed.  With equal spacing on every axis (ISO) one
  // coefficient per offset serves all axes: R pairs, kept in registers.
  constexpr bool PCOEF = ISO || R <= 6;
  constexpr int NPC = PCOEF ? R : 1;
  const float2 c0v = make_float2(p.c0, p.c0);
  float2 cxv[NPC], cyv[ISO ? 1 : NPC], czv[!ISO && PCOEF && RZ > 0 ? RZ : 1];
#pragma unroll
  for (int k = 0; k < NPC; ++k) cxv[k] = make_float2(p.cx[k], p.cx[k]);
#pragma unroll
  for (int k = 0; k < (ISO ? 0 : NPC); ++k) cyv[k] = make_float2(p.cy[k], p.cy[k]);
#pragma unroll
  for (int k = 0; k < (!ISO && PCOEF ? RZ : 0); ++k) czv[k] = make_float2(p.cz[k], p.cz[k]);
  // acc += c_{axis,k} * (a + b) on a packed pair (axis 0 = x, 1 = axis 1, 2 = axis 2);
  // anisotropic spacing only
  auto tap2 = [&](float2& acc, int axis, int k, const float2& a, const float2& b) {
    const float2 sum = __fadd2_rn(a, b);
    if constexpr (PCOEF) {
      acc = __ffma2_rn(axis == 0 ? cxv[k] : (axis == 1 ? cyv[k] : czv[k]), sum, acc);
    } else {
      const float cs = axis == 0 ? p.cx[k] : (axis == 1 ? p.cy[k] : p.cz[k]);
      acc.x = fmaf(cs, sum.x, acc.x);
      acc.y = fmaf(cs, sum.y, acc.y);
    }
  };

  // Register queue of the centre level along the streamed axis.  Planes are
  // processed in groups of QU: before a group starting at output plane z,
  // q[0 .. 2RZ-1] hold planes z-RZ .. z+RZ-1; plane z+u+RZ of the group lands
  // in q[2RZ+u], and the queue moves down by QU after the group (by one after
  // a single plane).  With UR > 1 (QU = 1) a group of UR planes renames the
  // queue instead of moving it: output plane u of the group reads the plane at
  // offset i of its window from q[(u + i) % NQ], and after the group the queue
  // is rotated once by UR (no move at all when UR = NQ).
  constexpr int QU = L::QU;
  constexpr int NQ = 2 * RZ + QU;
  constexpr int UR = L::UR;
  static_assert(UR == 1 || QU == 1, "renamed groups take one plane per queue slot");
  float4 q[NQ];
#pragma unroll
  for (int i = 0; i < NQ; ++i) q[i] = make_float4(0.f, 0.f, 0.f, 0.f);

  bool ok = true;
  if constexpr (L::DIRECT_FILL) {
    // the first 2RZ queue planes (z0 - RZ .. z0 + RZ - 1) straight from the
    // centre level, all loads in flight at once: zero outside the grid like
    // the tile loads' out-of-bounds fill (columns from NX to the pitch hold
    // zeros in every field slot)
    const float* cur = p.fields + p.cur * p.slot_elems;
    const bool col = gy < p.NY && gx < p.pitch;
    const long long plane = static_cast<long long>(p.NY) * p.pitch;
    const long long at = static_cast<long long>(gy) * p.pitch + gx;
#pragma unroll
    for (int s = 0; s < 2 * RZ; ++s) {
      const int z = z0 - RZ + s;
      q[s] = (col && z >= 0 && z < p.NZ) ? __ldg(reinterpret_cast<const float4*>(cur + z * plane + at))
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  } else {
#pragma unroll
    for (int s = 0; s < 2 * RZ; ++s) {
      const int slot = s % L::NSU;
      ok = mbar_wait_bounded(&fullU[slot], (s / L::NSU) & 1, abort_flag, p.wait_ns);
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      q[s] = lds4(Ubase + slot * (L::Q_STRIDE / 4) + qofs);
      if (L::LEAD || s < RZ) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&emptyU[slot]);
      }
    }
  }
  // ring sequence of output plane 0's stage
  constexpr int S0 = L::DIRECT_FILL ? 0 : 2 * RZ;

  const long long plane_elems = static_cast<long long>(p.NY) * p.pitch;
  long long idx = static_cast<long long>(z0) * plane_elems + static_cast<long long>(gy) * p.pitch + gx;
  // 16-bit snapshots read by the imaging condition: this thread's slab scale
  // for plane z0 + j is scale_ptr[j * scale_plane], prefetched a plane ahead
  const long long scale_plane = static_cast<long long>(p.slabs_y) * p.slabs_x;
  const float* scale_ptr = nullptr;
  float scale_next = 1.f;
  if constexpr (mode_is_grad(MODE) && FMT != 0) {
    scale_ptr = p.scale_in + (static_cast<long long>(z0) * p.slabs_y + (min(gy, p.NY - 1) >> 1)) * p.slabs_x + bx;
    scale_next = __ldg(scale_ptr);
  }
  float* const out_base = p.fields + p.prev * p.slot_elems;
  int j = 0;
  // ring positions of output plane j: plane z+R has sequence j+S0 in the
  // queue-feed ring, the centre plane j+S0-RZ, the per-point tiles j
  int ring_un = S0 % L::NSU, ring_ps = 0;
  uint32_t phase_un = (S0 / L::NSU) & 1, phase_ps = 0;

  // One output plane z = z0 + j, taking its queue entries at offset O of a
  // window renamed by PH (entry i at q[(PH + O + i) % NQ]).
  // un / pu: queue-feed stage and phase of the plane; ps / pp: its per-point
  // stage and phase (the same stage in the one-ring layout)
  auto plane = [&](auto oc, auto phc, int un, uint32_t pu, int ps, uint32_t pp) -> bool {
    constexpr int O = decltype(oc)::value;
    constexpr int PH = decltype(phc)::value;
    auto qi = [](int i) { return (PH + O + i) % NQ; };
    const int uc = un >= RZ ? un - RZ : un + L::NSU - RZ;  // slot of the centre plane
    bool good = mbar_wait_bounded(&fullU[un], pu, abort_flag, p.wait_ns);
    if (!__all_sync(0xffffffffu, good)) return false;
    q[qi(2 * RZ)] = lds4(Ubase + un * (L::Q_STRIDE / 4) + qofs);
    if constexpr (L::LEAD && !L::COMBINED) {
      __syncwarp();
      if (lane == 0) mbar_arrive(&emptyU[un]);
    }
    const float4 c = q[qi(RZ)];
    if constexpr (L::LEAD && !L::COMBINED) {
      // the centre halo box arrives with the per-point tiles
      good = mbar_wait_bounded(&fullP[ps], pp, abort_flag, p.wait_ns);
      if (!__all_sync(0xffffffffu, good)) return false;
    }
    const float* Uc = L::LEAD ? reinterpret_cast<const float*>(Pbase + ps * L::P_BYTES + L::HALO_OFF) + lofs
                              : Ubase + uc * (L::Q_STRIDE / 4) + lofs;

    // Laplacian on two packed pairs (points 0,1 and 2,3 of the quad)
    float2 la = __fmul2_rn(c0v, make_float2(c.x, c.y));
    float2 lb = __fmul2_rn(c0v, make_float2(c.z, c.w));
    if constexpr (ISO) {
      // one coefficient per offset k: the axis-2 and axis-1 neighbour pairs
      // at distance k are summed before a single multiply
#pragma unroll
      for (int k = 1; k <= R; ++k) {
        const float4 ya = lds4(Uc - k * T::UW);
        const float4 yb = lds4(Uc + k * T::UW);
        float2 sa = __fadd2_rn(make_float2(ya.x, ya.y), make_float2(yb.x, yb.y));
        float2 sb = __fadd2_rn(make_float2(ya.z, ya.w), make_float2(yb.z, yb.w));
        if constexpr (RZ > 0) {
          const float4 za = q[qi(RZ - k)];
          const float4 zb = q[qi(RZ + k)];
          sa = __fadd2_rn(sa, __fadd2_rn(make_float2(za.x, za.y), make_float2(zb.x, zb.y)));
          sb = __fadd2_rn(sb, __fadd2_rn(make_float2(za.z, za.w), make_float2(zb.z, zb.w)));
        }
        if constexpr (PCOEF) {
          la = __ffma2_rn(cxv[k - 1], sa, la);
          lb = __ffma2_rn(cxv[k - 1], sb, lb);
        } else {
          la.x = fmaf(p.cx[k - 1], sa.x, la.x);
          la.y = fmaf(p.cx[k - 1], sa.y, la.y);
          lb.x = fmaf(p.cx[k - 1], sb.x, lb.x);
          lb.y = fmaf(p.cx[k - 1], sb.y, lb.y);
        }
      }
    } else {
#pragma unroll
      for (int k = 1; k <= RZ; ++k) {
        const float4 a = q[qi(RZ - k)];
        const float4 b = q[qi(RZ + k)];
        tap2(la, 2, k - 1, make_float2(a.x, a.y), make_float2(b.x, b.y));
        tap2(lb, 2, k - 1, make_float2(a.z, a.w), make_float2(b.z, b.w));
      }
#pragma unroll
      for (int k = 1; k <= R; ++k) {
        const float4 a = lds4(Uc - k * T::UW);
        const float4 b = lds4(Uc + k * T::UW);
        tap2(la, 1, k - 1, make_float2(a.x, a.y), make_float2(b.x, b.y));
        tap2(lb, 1, k - 1, make_float2(a.z, a.w), make_float2(b.z, b.w));
      }
    }
    {
      constexpr int NH = T::HX / 4;  // halo quads per side
      float v[4 + 2 * T::HX];
#pragma unroll
      for (int k = 0; k < NH; ++k) {
        const float4 l = lds4(Uc - 4 * (k + 1));
        const float4 r = lds4(Uc + 4 * (k + 1));
        v[T::HX - 4 * (k + 1) + 0] = l.x;
        v[T::HX - 4 * (k + 1) + 1] = l.y;
        v[T::HX - 4 * (k + 1) + 2] = l.z;
        v[T::HX - 4 * (k + 1) + 3] = l.w;
        v[T::HX + 4 * (k + 1) + 0] = r.x;
        v[T::HX + 4 * (k + 1) + 1] = r.y;
        v[T::HX + 4 * (k + 1) + 2] = r.z;
        v[T::HX + 4 * (k + 1) + 3] = r.w;
      }
      v[T::HX + 0] = c.x;
      v[T::HX + 1] = c.y;
      v[T::HX + 2] = c.z;
      v[T::HX + 3] = c.w;
#pragma unroll
      for (int k = 1; k <= R; ++k) {
        constexpr int H = T::HX;
        if (k % 2 == 0) {
          // even offsets keep the pairs register-aligned
          tap2(la, 0, k - 1, make_float2(v[H - k], v[H + 1 - k]), make_float2(v[H + k], v[H + 1 + k]));
          tap2(lb, 0, k - 1, make_float2(v[H + 2 - k], v[H + 3 - k]), make_float2(v[H + 2 + k], v[H + 3 + k]));
        } else {
          la.x = fmaf(p.cx[k - 1], v[H + 0 - k] + v[H + 0 + k], la.x);
          la.y = fmaf(p.cx[k - 1], v[H + 1 - k] + v[H + 1 + k], la.y);
          lb.x = fmaf(p.cx[k - 1], v[H + 2 - k] + v[H + 2 + k], lb.x);
          lb.y = fmaf(p.cx[k - 1], v[H + 3 - k] + v[H + 3 + k], lb.y);
        }
      }
    }
    if constexpr (!L::LEAD) {
      good = mbar_wait_bounded(&fullP[ps], pp, abort_flag, p.wait_ns);
      if (!__all_sync(0xffffffffu, good)) return false;
    }
    const unsigned char* Pst = Pbase + ps * L::P_BYTES;
    const float4 prev = *reinterpret_cast<const float4*>(Pst + L::PREV_OFF + tofs);
    const float4 cm = *reinterpret_cast<const float4*>(Pst + L::CM_OFF + tofs);
    if constexpr (MODE == MODE_SRC) {
      // source field of the scattered wavefield enters like the Laplacian
      const float4 src = *reinterpret_cast<const float4*>(Pst + L::G_OFF + tofs);
      la = __fadd2_rn(la, make_float2(src.x, src.y));
      lb = __fadd2_rn(lb, make_float2(src.z, src.w));
    }

    const int gz = z0 + j;
    const float ez = NDIM == 3 ? sponge_term(gz, p.NZ, p.nblz, p.emz) : 0.f;
    float4 out;
    if (sponge_sum(exy_max, ez) == 0.f) {
      // undamped: new = 2 cur - prev + cm L (the damped formula at k = 0), on
      // packed pairs
      const float2 m1 = make_float2(-1.f, -1.f);
      const float2 ca = make_float2(c.x, c.y), cb = make_float2(c.z, c.w);
      const float2 oa = __ffma2_rn(make_float2(cm.x, cm.y), la,
                                   __ffma2_rn(m1, make_float2(prev.x, prev.y), __fadd2_rn(ca, ca)));
      const float2 ob = __ffma2_rn(make_float2(cm.z, cm.w), lb,
                                   __ffma2_rn(m1, make_float2(prev.z, prev.w), __fadd2_rn(cb, cb)));
      out = make_float4(oa.x, oa.y, ob.x, ob.y);
    } else if constexpr (L::PACKED_DAMP) {
      // damped, on packed pairs: the operations of damp_inv and of the update
      // below, each rounded once, so the same values as one point at a time
      const float2 hv = make_float2(p.half_inv_dt, p.half_inv_dt);
      const float2 one = make_float2(1.f, 1.f);
      auto damped = [&](float ea, float eb, float2 cmv, float2 lv, float2 pv, float2 cv) -> float2 {
        const float2 eta = make_float2(sponge_sum(ea, ez), sponge_sum(eb, ez));
        const float2 k = __fmul2_rn(__fmul2_rn(eta, cmv), hv);
        const float2 omk = __fadd2_rn(one, make_float2(-k.x, -k.y));
        const float2 d = __fadd2_rn(one, k);
        const float2 inv =
            make_float2(eta.x == 0.f ? 1.f : __fdividef(1.f, d.x), eta.y == 0.f ? 1.f : __fdividef(1.f, d.y));
        const float2 t = __ffma2_rn(make_float2(-omk.x, -omk.y), pv, __fadd2_rn(cv, cv));
        return __fmul2_rn(__ffma2_rn(cmv, lv, t), inv);
      };
      const float2 oa = damped(exy[0], exy[1], make_float2(cm.x, cm.y), la, make_float2(prev.x, prev.y),
                               make_float2(c.x, c.y));
      const float2 ob = damped(exy[2], exy[3], make_float2(cm.z, cm.w), lb, make_float2(prev.z, prev.w),
                               make_float2(c.z, c.w));
      out = make_float4(oa.x, oa.y, ob.x, ob.y);
    } else {
      float omk;
      float inv = damp_inv(sponge_sum(exy[0], ez), cm.x, p.half_inv_dt, omk);
      out.x = fmaf(cm.x, la.x, fmaf(-omk, prev.x, 2.f * c.x)) * inv;
      inv = damp_inv(sponge_sum(exy[1], ez), cm.y, p.half_inv_dt, omk);
      out.y = fmaf(cm.y, la.y, fmaf(-omk, prev.y, 2.f * c.y)) * inv;
      inv = damp_inv(sponge_sum(exy[2], ez), cm.z, p.half_inv_dt, omk);
      out.z = fmaf(cm.z, lb.x, fmaf(-omk, prev.z, 2.f * c.z)) * inv;
      inv = damp_inv(sponge_sum(exy[3], ez), cm.w, p.half_inv_dt, omk);
      out.w = fmaf(cm.w, lb.y, fmaf(-omk, prev.w, 2.f * c.w)) * inv;
    }
    if (store_ok) *reinterpret_cast<float4*>(out_base + idx) = out;

    if constexpr (mode_is_snap(MODE)) {
      if constexpr (FMT == 0) {
        if (store_ok) store_snap4<0>(p.snap_out, idx, c, 1.f);
      } else {
        // slab max |u|: non-negative floats order like their bit patterns, so
        // one integer warp reduction gives it
        const float lmax = fmaxf(fmaxf(fabsf(c.x), fabsf(c.y)), fmaxf(fabsf(c.z), fabsf(c.w)));
        const float amax = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(lmax)));
        const float s = slab_scale(amax);
        if (store_ok) store_snap4<FMT>(p.snap_out, idx, c, slab_inv_scale(s));
        if (lane == 0 && gy < p.NY)
          p.scale_out[(static_cast<long long>(gz) * p.slabs_y + (gy >> 1)) * p.slabs_x + bx] = s;
      }
    }
    if constexpr (MODE == MODE_BORN_SRC) {
      // Born source of the scattered field: -dm (new - 2 cur + prev) / dt^2
      const float4 dm = *reinterpret_cast<const float4*>(Pst + L::G_OFF + tofs);
      float4 sb;
      sb.x = -dm.x * (out.x - 2.f * c.x + prev.x) * p.inv_dt2;
      sb.y = -dm.y * (out.y - 2.f * c.y + prev.y) * p.inv_dt2;
      sb.z = -dm.z * (out.z - 2.f * c.z + prev.z) * p.inv_dt2;
      sb.w = -dm.w * (out.w - 2.f * c.w + prev.w) * p.inv_dt2;
      if (store_ok) *reinterpret_cast<float4*>(p.grad + idx) = sb;
    }
    if constexpr (mode_is_grad(MODE)) {
      float s = 1.f;
      if constexpr (FMT != 0) {
        // slab scale of this plane was loaded one plane ahead
        s = scale_next;
        if (j + 1 < nP) scale_next = __ldg(scale_ptr + (j + 1) * scale_plane);
      }
      const float4 u = load_snap4_smem<FMT>(Pst + L::S_OFF + (ty * T::BX + 4 * tx) * L::SNAP_ELEM, s);
      float4 g = *reinterpret_cast<const float4*>(Pst + L::G_OFF + tofs);
      g.x -= u.x * (out.x - 2.f * c.x + prev.x) * p.inv_dt2;
      g.y -= u.y * (out.y - 2.f * c.y + prev.y) * p.inv_dt2;
      g.z -= u.z * (out.z - 2.f * c.z + prev.z) * p.inv_dt2;
      g.w -= u.w * (out.w - 2.f * c.w + prev.w) * p.inv_dt2;
      if (store_ok) *reinterpret_cast<float4*>(p.grad + idx) = g;
    }

    __syncwarp();
    if (lane == 0) {
      if constexpr (L::COMBINED) {
        mbar_arrive(&emptyU[un]);
      } else {
        if constexpr (!L::LEAD) mbar_arrive(&emptyU[uc]);
        mbar_arrive(&emptyP[ps]);
      }
    }
    return true;
  };
  // the plane at the runtime ring positions
  auto ring = [&](auto oc, auto phc) -> bool {
    if constexpr (L::COMBINED) return plane(oc, phc, ring_un, phase_un, ring_un, phase_un);
    else return plane(oc, phc, ring_un, phase_un, ring_ps, phase_ps);
  };

  // ring slots and phases advance by one per plane (no division in the loop)
  auto advance = [&]() {
    ++j;
    idx += plane_elems;
    if (++ring_un == L::NSU) {
      ring_un = 0;
      phase_un ^= 1u;
    }
    if (++ring_ps == L::NSP) {
      ring_ps = 0;
      phase_ps ^= 1u;
    }
  };
  if (ok && QU == 2) {
    while (j + 2 <= nP) {
      ok = ring(IntC<0>{}, IntC<0>{});
      if (!ok) break;
      advance();
      ok = ring(IntC<QU - 1>{}, IntC<0>{});
      if (!ok) break;
      advance();
#pragma unroll
      for (int i = 0; i < 2 * RZ; ++i) q[i] = q[i + QU];
    }
  }
  if constexpr (UR > 1 && L::COMBINED && UR == L::NSU) {
    // groups of NSU planes from j = 0: plane u of a group uses stage
    // (2RZ + u) % NSU, whose phase is the group's parity flipped by
    // (2RZ + u) / NSU -- both known at compile time but for the parity
    uint32_t gpar = 0;
    auto renamed = [&](auto phc) -> bool {
      constexpr int u = decltype(phc)::value;
      constexpr int sl = (S0 + u) % L::NSU;
      const uint32_t par = gpar ^ static_cast<uint32_t>(((S0 + u) / L::NSU) & 1);
      if (!plane(IntC<0>{}, phc, sl, par, sl, par)) return false;
      ++j;
      idx += plane_elems;
      return true;
    };
    while (ok && j + UR <= nP) {
      ok = call_in_order(renamed, IntC<0>{}, IntC<UR>{});
      if (!ok) break;
      gpar ^= 1u;
      if constexpr (UR % NQ != 0) {
        float4 t[NQ];
#pragma unroll
        for (int i = 0; i < NQ; ++i) t[i] = q[(i + UR) % NQ];
#pragma unroll
        for (int i = 0; i < NQ; ++i) q[i] = t[i];
      }
    }
    ring_un = (j + S0) % L::NSU;
    phase_un = ((j + S0) / L::NSU) & 1;
  } else if constexpr (UR > 1) {
    auto renamed = [&](auto phc) -> bool {
      if (!ring(IntC<0>{}, phc)) return false;
      advance();
      return true;
    };
    while (ok && j + UR <= nP) {
      ok = call_in_order(renamed, IntC<0>{}, IntC<UR>{});
      if (!ok) break;
      if constexpr (UR % NQ != 0) {
        float4 t[NQ];
#pragma unroll
        for (int i = 0; i < NQ; ++i) t[i] = q[(i + UR) % NQ];
#pragma unroll
        for (int i = 0; i < NQ; ++i) q[i] = t[i];
      }
    }
  }
  if (ok) {
    while (j < nP) {
      ok = ring(IntC<0>{}, IntC<0>{});
      if (!ok) break;
      advance();
#pragma unroll
      for (int i = 0; i < 2 * RZ; ++i) q[i] = q[i + 1];
    }
  }
  if (!ok && lane == 0) {
    *abort_flag = 1;
    atomicExch(p.status, kDevTimeout);
  }
}

template <int R, int NDIM, int MODE, bool ISO>
__global__ void __launch_bounds__(StepTraits<R, NDIM, ISO>::NTHREADS, (StepLayout<R, NDIM, MODE, ISO>::MIN_BLOCKS))
    step_kernel(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_p,
                const __grid_constant__ CUtensorMap tm_cm, const __grid_constant__ CUtensorMap tm_g,
                const __grid_constant__ CUtensorMap tm_s, const StepParams p) {
  const int z0 = static_cast<int>(blockIdx.z) * p.zchunk;
  step_body<R, NDIM, MODE, ISO>(tm_u, tm_p, tm_cm, tm_g, tm_s, p, blockIdx.x, blockIdx.y, z0, min(z0 + p.zchunk, p.NZ));
}

// Receiver sampling of row n from the centre level by the consumer threads of
// one CTA (share [r0, r1) of the points), with the lane layout and the
// reduction of gather_kernel: 8 lanes per point, one corner each, summed by
// xor shuffles.  Whole warps take part in every round; the loads of KR rounds
// are issued before any of their values is used, so that a CTA's share costs
// a few memory latencies, hidden behind the loads of its first planes.
template <int NCW, int KR>
__device__ __forceinline__ void sample_share(const GatherSet& gs, const float* __restrict__ field, float* out,
                                             long long r0, long long r1, int ctid) {
  constexpr int STRIDE = NCW * 32;
  const int lane = ctid & 31;
  const int c = lane & 7;
  const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
  const long long lanes = (r1 - r0) * 8;
  for (long long t0 = static_cast<long long>(ctid - lane); t0 < lanes; t0 += KR * STRIDE) {
    float w[KR], v[KR];
    long long at[KR];
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      const long long t = t0 + k * STRIDE + lane;
      w[k] = 0.f;
      at[k] = -1;
      if (t < lanes) {
        const long long pt = r0 + (t >> 3);
        const float fx = gs.frac[3 * pt], fy = gs.frac[3 * pt + 1], fz = gs.frac[3 * pt + 2];
        float wk = (cx ? fx : 1.f - fx) * (cy ? fy : 1.f - fy);
        wk *= (cz ? fz : 1.f - fz);
        w[k] = wk;
        at[k] = gs.base[pt] + cx + cy * gs.sy + cz * gs.sz;
      }
    }
#pragma unroll
    for (int k = 0; k < KR; ++k) v[k] = at[k] >= 0 ? __fmul_rn(w[k], field[at[k]]) : 0.f;
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      float x = v[k];
      for (int off = 4; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
      const long long t = t0 + k * STRIDE + lane;
      if (t < lanes && c == 0) out[r0 + (t >> 3)] = x;
    }
  }
}

// Segmented plain step (3D, SegWork): CTA b computes its run of the tile-major
// column sequence, one step body per column it touches (the ring barriers are
// ended and initialised again in between), samples its share of the receivers
// from the centre level during its first segment, and then injects source row
// n into the cells of its segments.
template <int R, bool ISO>
__global__ void __launch_bounds__(StepTraits<R, 3, ISO>::NTHREADS, (StepLayout<R, 3, MODE_PLAIN, ISO>::MIN_BLOCKS))
    step_seg_kernel(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_p,
                    const __grid_constant__ CUtensorMap tm_cm, const __grid_constant__ CUtensorMap tm_g,
                    const __grid_constant__ CUtensorMap tm_s, const StepParams p, const SegWork w) {
  using T = StepTraits<R, 3, ISO>;
  using L = StepLayout<R, 3, MODE_PLAIN, ISO>;
  const long long g0 = w.run_start[blockIdx.x];
  const long long g1 = w.run_start[blockIdx.x + 1];
  bool first = true;
  auto pre = [&](int ctid) {
    if (!first || w.rec_out == nullptr) return;
    const long long share = (w.rec.n + gridDim.x - 1) / gridDim.x;
    const long long r0 = min(static_cast<long long>(blockIdx.x) * share, w.rec.n);
    const long long r1 = min(r0 + share, w.rec.n);
    sample_share<T::NCW, (T::NCW == 8 && R >= 5) ? 4 : 8>(w.rec, p.fields + p.cur * p.slot_elems, w.rec_out, r0, r1, ctid);
  };
  for (long long g = g0; g < g1;) {
    const long long col = g / p.NZ;
    const int z0 = static_cast<int>(g - col * p.NZ);
    const int z1 = static_cast<int>(min(static_cast<long long>(p.NZ), z0 + (g1 - g)));
    if (!first) {
      // every thread is done with the previous segment's ring
      __syncthreads();
      if (threadIdx.x == 0) {
        extern __shared__ unsigned char smem_raw[];
        uint64_t* bars = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) &
                                                     ~static_cast<uintptr_t>(127));
        for (int i = 0; i < 2 * (L::NSU + L::NSP); ++i) mbar_inval(&bars[i]);
      }
    }
    step_body<R, 3, MODE_PLAIN, ISO>(tm_u, tm_p, tm_cm, tm_g, tm_s, p, static_cast<int>(col % w.tiles_x),
                                     static_cast<int>(col / w.tiles_x), z0, z1, pre);
    first = false;
    g += z1 - z0;
  }
  if (w.inj_vals == nullptr) return;
  // the new level of the CTA's cells is written; the arithmetic of inject_kernel
  __syncthreads();
  float* field = p.fields + p.prev * p.slot_elems;
  for (int e = w.inj_ptr[blockIdx.x] + static_cast<int>(threadIdx.x); e < w.inj_ptr[blockIdx.x + 1];
       e += blockDim.x) {
    const int k = w.inj_list[e];
    float s = 0.f;
    for (int i = w.inj.rowptr[k]; i < w.inj.rowptr[k + 1]; ++i) s = fmaf(w.inj.w[i], w.inj_vals[w.inj.pidx[i]], s);
    field[w.inj.cell[k]] = fmaf(w.inj.coef[k], s, field[w.inj.cell[k]]);
  }
}

}  // namespace dev

}  // namespace wave
