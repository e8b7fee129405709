// Two leapfrog levels per pass over memory (temporal blocking; the paper lists
// time tiling as future work in Sec. VI and doubts it because sparse
// operators sit inside the time loop).  From u^{n-1}, u^n and cm = dt^2/m one
// launch produces u^{n+1} and u^{n+2} of Listing 1 / Eq. 1,
//   u^{k+1} = (2 u^k - (1 - k_eta) u^{k-1} + cm L(u^k)) / (1 + k_eta),
// reading three fields and writing two: 10 bytes of HBM traffic per point
// update instead of the 16 of the single-level step.  No source is injected
// between the two levels, so the pass serves source-free propagation (an
// initial-value problem); receivers are sampled from both output levels
// afterwards.
//
// Order 8 (radius 4), 3D.  A CTA owns a 64 x 16 column tile of level n+2 and
// streams a chunk of planes.  Stage 1 computes level n+1 on the tile widened
// by 4 points in x and R rows in y (72 x 24 columns, one quad of 4 x points
// per consumer thread: 432 threads), from a register queue of level n along z
// and a TMA-loaded halo box of level n (80 x 32); it runs R planes ahead of
// stage 2 and over R extra planes at each end of the chunk, so the halo of
// level n+1 is recomputed rather than exchanged.  Its planes go to a shared
// ring of 2R + 2 planes.  Stage 2 computes level n+2 on the tile, reading
// every tap of level n+1 from that ring, level n at its plane from the stage-1
// queue and cm from a small ring written by stage 1.  Level n+1 outside the
// grid is zero (the zero ghost of the single-level step).  Loads of level n,
// n-1 and cm go through the producer warp shared with step_kernel
// (produce<>, lead-plane layout) at shifted coordinates.  A CTA-wide mbarrier
// with a bounded wait separates the stages of a plane, so a warp that takes
// the timeout path cannot leave the others waiting without limit.
#include <atomic>

#include "step_kernel.cuh"

namespace wave {
namespace dev {

template <int R>
struct Step2Layout {
  static_assert(R >= 1 && R <= 4, "two-level pass: the x extension of 4 points covers radius <= 4");
  static constexpr int BX = 64, BY = 16;      // level n+2 outputs per CTA
  static constexpr int H1 = 4;                // x extension of level n+1 (whole quads, >= R)
  static constexpr int EX = BX + 2 * H1;      // 72 columns of level n+1
  static constexpr int EY = BY + 2 * R;       // rows of level n+1
  static constexpr int HX = 4;                // x halo of level n around the extended tile
  static constexpr int RZ = R;
  static constexpr int UW = EX + 2 * HX;      // 80
  static constexpr int UH = EY + 2 * R;
  static constexpr int EQ = EX / 4;           // quads per extended row
  static constexpr int NWORK = EQ * EY;       // consumer threads owning a column
  static constexpr int NCW = (NWORK + 31) / 32;
  static constexpr int NTHREADS = (NCW + 1) * 32;
  static constexpr int E_BYTES = EX * EY * 4;  // one extended plane
  static constexpr int U_BYTES = UW * UH * 4;
  static constexpr int U_STRIDE = (U_BYTES + 127) / 128 * 128;
  static constexpr bool LEAD = true;
  static constexpr bool COMBINED = false;  // separate queue-feed and per-point barriers
  static constexpr int PF = 3;
  static constexpr int NSU = PF + 1;
  static constexpr int NSP = PF + 1;
  static constexpr int Q_BYTES = E_BYTES;
  static constexpr int Q_STRIDE = (E_BYTES + 127) / 128 * 128;
  static constexpr int HALO_OFF = 0;
  static constexpr int PREV_OFF = U_STRIDE;
  static constexpr int CM_OFF = PREV_OFF + Q_STRIDE;
  static constexpr int G_OFF = CM_OFF + Q_STRIDE;  // no third tile in this pass
  static constexpr int S_OFF = G_OFF;
  static constexpr int P_TX = U_BYTES + 2 * E_BYTES;
  static constexpr int P_BYTES = U_STRIDE + 2 * Q_STRIDE;
  static constexpr int NB1 = 2 * R + 2;       // ring of level n+1 planes
  static constexpr int C_BYTES = BX * BY * 4;
  static constexpr int NC = R + 2;            // ring of cm planes of the output tile
  static constexpr int NQ = 2 * R + 1;
  static constexpr int UR = 3;                // planes per renamed register-queue group
  static constexpr int BAR_BYTES = ((16 * (NSU + NSP) + 16 + 16 + 127) / 128) * 128;
  static constexpr int U_OFF = BAR_BYTES;
  static constexpr int PST_OFF = U_OFF + NSU * Q_STRIDE;
  static constexpr int B1_OFF = PST_OFF + NSP * P_BYTES;
  static constexpr int C_OFF = B1_OFF + NB1 * Q_STRIDE;
  static constexpr int SMEM = C_OFF + NC * C_BYTES + 128;
  static_assert(SMEM <= 227 * 1024, "two-level pass exceeds the shared memory of one CTA");
  static_assert(P_BYTES % 128 == 0 && Q_STRIDE % 128 == 0, "stages keep 128-byte alignment");
};

template <int R>
__global__ void __launch_bounds__(Step2Layout<R>::NTHREADS, 1)
    step2_kernel(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_e,
                 const __grid_constant__ CUtensorMap tm_cm, const StepParams p) {
  using L = Step2Layout<R>;
  constexpr int NQ = L::NQ;
  constexpr int UW = L::UW;
  constexpr int EX = L::EX;

  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
  uint64_t* fullU = reinterpret_cast<uint64_t*>(smem);
  uint64_t* emptyU = fullU + L::NSU;
  uint64_t* fullP = emptyU + L::NSU;
  uint64_t* emptyP = fullP + L::NSP;
  uint64_t* stage_bar = emptyP + L::NSP;  // stage 1 of a plane done by every consumer warp
  volatile int* abort_flag = reinterpret_cast<volatile int*>(stage_bar + 1);
  float* Ubase = reinterpret_cast<float*>(smem + L::U_OFF);
  unsigned char* Pbase = smem + L::PST_OFF;
  float* B1 = reinterpret_cast<float*>(smem + L::B1_OFF);
  float* Cring = reinterpret_cast<float*>(smem + L::C_OFF);

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int x0 = blockIdx.x * L::BX;
  const int y0 = blockIdx.y * L::BY;
  const int z0 = blockIdx.z * p.zchunk;
  const int z1 = min(z0 + p.zchunk, p.NZ);
  const int nP = z1 - z0;
  if (nP <= 0) return;
  const int nS = nP + 2 * R;  // stage-1 planes z0 - R .. z1 + R - 1
  const int ex0 = x0 - L::H1, ey0 = y0 - R;

  if (tid == 0) {
    for (int i = 0; i < L::NSU; ++i) {
      mbar_init(&fullU[i], 1);
      mbar_init(&emptyU[i], L::NCW);
    }
    for (int i = 0; i < L::NSP; ++i) {
      mbar_init(&fullP[i], 1);
      mbar_init(&emptyP[i], L::NCW);
    }
    mbar_init(stage_bar, L::NCW);
    *abort_flag = 0;
    fence_mbarrier_init();
  }
  __syncthreads();

  if (warp == L::NCW) {
    // queue boxes of level n for planes z0 - 2R .., per-point stages (level-n
    // halo box, level n-1 and cm on the extended tile) for planes z0 - R ..
    produce<L, R, MODE_PLAIN>(tm_u, tm_e, tm_cm, tm_cm, tm_e, p, ex0, ey0, z0 - R, nS + 2 * R, fullU, emptyU, fullP,
                              emptyP, abort_flag, Ubase, Pbase);
    return;
  }
  // ------------------------------------------------------------------ consumers
  const bool work = tid < L::NWORK;
  const int eq = work ? tid % L::EQ : 0;   // quad of the extended row
  const int er = work ? tid / L::EQ : 0;   // extended row
  const int gx = ex0 + 4 * eq;
  const int gy = ey0 + er;
  const bool interior = work && eq >= 1 && eq <= L::EQ - 2 && er >= R && er < R + L::BY;
  const bool row_in = gy >= 0 && gy < p.NY;
  const bool store_ok = interior && gx < p.NX && gy < p.NY;
  const int lofs = (R + er) * UW + L::HX + 4 * eq;  // quad in the level-n halo box
  const int eofs = er * EX + 4 * eq;                // quad in an extended plane
  const int cofs = (er - R) * L::BX + 4 * (eq - 1); // quad in an output-tile plane (interior)

  // level n+1 is zero outside the grid: mask per x point
  float xmask[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) xmask[i] = (gx + i >= 0 && gx + i < p.NX && row_in) ? 1.f : 0.f;
  float ex[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) ex[i] = sponge_term(gx + i, p.NX, p.nblx, p.emx);
  const float ey = sponge_term(gy, p.NY, p.nbly, p.emy);
  float exy[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) exy[i] = sponge_sum(ex[i], ey);
  const float exy_max = fmaxf(fmaxf(exy[0], exy[1]), fmaxf(exy[2], exy[3]));

  float2 cxv[R], cyv[R], czv[R];
#pragma unroll
  for (int k = 0; k < R; ++k) {
    cxv[k] = make_float2(p.cx[k], p.cx[k]);
    cyv[k] = make_float2(p.cy[k], p.cy[k]);
    czv[k] = make_float2(p.cz[k], p.cz[k]);
  }
  const float2 c0v = make_float2(p.c0, p.c0);
  auto tap2 = [&](float2& acc, const float2& c, const float4& a, const float4& b, bool high) {
    const float2 s = high ? __fadd2_rn(make_float2(a.z, a.w), make_float2(b.z, b.w))
                          : __fadd2_rn(make_float2(a.x, a.y), make_float2(b.x, b.y));
    acc = __ffma2_rn(c, s, acc);
  };
  // x and axis-1 taps of a quad at `Uc` in a plane of row width W (floats);
  // axis-2 taps and the centre are added by the caller
  auto xy_taps = [&](const float* Uc, int W, const float4& c, float2& la, float2& lb) {
#pragma unroll
    for (int k = 1; k <= R; ++k) {
      const float4 a = lds4(Uc - k * W);
      const float4 b = lds4(Uc + k * W);
      tap2(la, cyv[k - 1], a, b, false);
      tap2(lb, cyv[k - 1], a, b, true);
    }
    const float4 l = lds4(Uc - 4);
    const float4 r = lds4(Uc + 4);
    const float v[12] = {l.x, l.y, l.z, l.w, c.x, c.y, c.z, c.w, r.x, r.y, r.z, r.w};
#pragma unroll
    for (int k = 1; k <= R; ++k) {
      if (k % 2 == 0) {
        la = __ffma2_rn(cxv[k - 1], __fadd2_rn(make_float2(v[4 - k], v[5 - k]), make_float2(v[4 + k], v[5 + k])), la);
        lb = __ffma2_rn(cxv[k - 1], __fadd2_rn(make_float2(v[6 - k], v[7 - k]), make_float2(v[6 + k], v[7 + k])), lb);
      } else {
        la.x = fmaf(p.cx[k - 1], v[4 - k] + v[4 + k], la.x);
        la.y = fmaf(p.cx[k - 1], v[5 - k] + v[5 + k], la.y);
        lb.x = fmaf(p.cx[k - 1], v[6 - k] + v[6 + k], lb.x);
        lb.y = fmaf(p.cx[k - 1], v[7 - k] + v[7 + k], lb.y);
      }
    }
  };
  // new level from centre c, Laplacian (la, lb), previous level and cm, with
  // the sponge of plane term ez
  auto update = [&](const float4& c, const float2& la, const float2& lb, const float4& prev, const float4& cm,
                    float ez) -> float4 {
    float4 out;
    if (sponge_sum(exy_max, ez) == 0.f) {
      const float2 m1 = make_float2(-1.f, -1.f);
      const float2 ca = make_float2(c.x, c.y), cb = make_float2(c.z, c.w);
      const float2 oa = __ffma2_rn(make_float2(cm.x, cm.y), la,
                                   __ffma2_rn(m1, make_float2(prev.x, prev.y), __fadd2_rn(ca, ca)));
      const float2 ob = __ffma2_rn(make_float2(cm.z, cm.w), lb,
                                   __ffma2_rn(m1, make_float2(prev.z, prev.w), __fadd2_rn(cb, cb)));
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
    return out;
  };

  // register queue of level n along axis 2 (stage 1), renamed over groups of
  // UR planes: window slot i of group plane u is a[(u + i) % NQ]
  float4 a[NQ];
#pragma unroll
  for (int i = 0; i < NQ; ++i) a[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  bool ok = true;
#pragma unroll
  for (int s = 0; s < 2 * R; ++s) {
    const int slot = s % L::NSU;
    ok = mbar_wait_bounded(&fullU[slot], (s / L::NSU) & 1, abort_flag, p.wait_ns);
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) break;
    a[s] = lds4(Ubase + slot * (L::Q_STRIDE / 4) + eofs);
    __syncwarp();
    if (lane == 0) mbar_arrive(&emptyU[slot]);
  }

  const long long plane_elems = static_cast<long long>(p.NY) * p.pitch;
  const long long col = static_cast<long long>(gy) * p.pitch + gx;  // used where store_ok
  float* const out1 = p.fields + p.out1 * p.slot_elems;
  float* const out2 = p.fields + p.out2 * p.slot_elems;
  int s = 0;                       // stage-1 plane z0 - R + s
  int ring_un = (2 * R) % L::NSU, ring_ps = 0;
  uint32_t phase_un = ((2 * R) / L::NSU) & 1, phase_ps = 0;
  int b1 = 0, cs = 0;              // ring slots of the current stage-1 plane

  auto plane = [&](auto phc) -> bool {
    constexpr int PH = decltype(phc)::value;
    auto qi = [](int i) { return (PH + i) % NQ; };
    const int pz = z0 - R + s;
    const int un = ring_un, ps = ring_ps;
    bool good = mbar_wait_bounded(&fullU[un], phase_un, abort_flag, p.wait_ns);
    if (!__all_sync(0xffffffffu, good)) return false;
    a[qi(2 * R)] = lds4(Ubase + un * (L::Q_STRIDE / 4) + eofs);
    __syncwarp();
    if (lane == 0) mbar_arrive(&emptyU[un]);
    good = mbar_wait_bounded(&fullP[ps], phase_ps, abort_flag, p.wait_ns);
    if (!__all_sync(0xffffffffu, good)) return false;
    const unsigned char* Pst = Pbase + ps * L::P_BYTES;

    // ---- stage 1: level n+1 at plane pz on the extended tile
    if (work) {
      const float4 c = a[qi(R)];
      float2 la = __fmul2_rn(c0v, make_float2(c.x, c.y));
      float2 lb = __fmul2_rn(c0v, make_float2(c.z, c.w));
#pragma unroll
      for (int k = 1; k <= R; ++k) {
        tap2(la, czv[k - 1], a[qi(R - k)], a[qi(R + k)], false);
        tap2(lb, czv[k - 1], a[qi(R - k)], a[qi(R + k)], true);
      }
      xy_taps(reinterpret_cast<const float*>(Pst + L::HALO_OFF) + lofs, UW, c, la, lb);
      const float4 prev = *reinterpret_cast<const float4*>(Pst + L::PREV_OFF + 4 * eofs);
      const float4 cm = *reinterpret_cast<const float4*>(Pst + L::CM_OFF + 4 * eofs);
      float4 v = update(c, la, lb, prev, cm, sponge_term(pz, p.NZ, p.nblz, p.emz));
      const bool plane_in = pz >= 0 && pz < p.NZ;
      v = make_float4(plane_in ? v.x * xmask[0] : 0.f, plane_in ? v.y * xmask[1] : 0.f,
                      plane_in ? v.z * xmask[2] : 0.f, plane_in ? v.w * xmask[3] : 0.f);
      *reinterpret_cast<float4*>(B1 + b1 * (L::Q_STRIDE / 4) + eofs) = v;
      if (interior) {
        *reinterpret_cast<float4*>(Cring + cs * (L::C_BYTES / 4) + cofs) = cm;
        if (store_ok && pz >= z0 && pz < z1)
          *reinterpret_cast<float4*>(out1 + static_cast<long long>(pz) * plane_elems + col) = v;
      }
    }
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&emptyP[ps]);
      mbar_arrive(stage_bar);
    }
    // every warp's stage-1 plane is in the rings before stage 2 reads them
    good = mbar_wait_bounded(stage_bar, s & 1, abort_flag, p.wait_ns);
    if (!__all_sync(0xffffffffu, good)) return false;

    // ---- stage 2: level n+2 at plane qz = pz - R on the output tile
    const int qz = pz - R;
    if (interior && s >= 2 * R) {
      const int bq = b1 >= R ? b1 - R : b1 + L::NB1 - R;  // ring slot of plane qz
      const float* Bq = B1 + bq * (L::Q_STRIDE / 4) + eofs;
      const float4 c = *reinterpret_cast<const float4*>(Bq);
      float2 la = __fmul2_rn(c0v, make_float2(c.x, c.y));
      float2 lb = __fmul2_rn(c0v, make_float2(c.z, c.w));
#pragma unroll
      for (int k = 1; k <= R; ++k) {
        const int lo = bq >= k ? bq - k : bq + L::NB1 - k;
        const int hi = bq + k < L::NB1 ? bq + k : bq + k - L::NB1;
        const float4 zl = lds4(B1 + lo * (L::Q_STRIDE / 4) + eofs);
        const float4 zh = lds4(B1 + hi * (L::Q_STRIDE / 4) + eofs);
        tap2(la, czv[k - 1], zl, zh, false);
        tap2(lb, czv[k - 1], zl, zh, true);
      }
      xy_taps(Bq, EX, c, la, lb);
      const int cq = cs >= R ? cs - R : cs + L::NC - R;
      const float4 cm = *reinterpret_cast<const float4*>(Cring + cq * (L::C_BYTES / 4) + cofs);
      const float4 prev = a[qi(0)];  // level n at plane qz
      const float4 v = update(c, la, lb, prev, cm, sponge_term(qz, p.NZ, p.nblz, p.emz));
      if (store_ok) *reinterpret_cast<float4*>(out2 + static_cast<long long>(qz) * plane_elems + col) = v;
    }
    return true;
  };
  auto advance = [&]() {
    ++s;
    if (++ring_un == L::NSU) {
      ring_un = 0;
      phase_un ^= 1u;
    }
    if (++ring_ps == L::NSP) {
      ring_ps = 0;
      phase_ps ^= 1u;
    }
    if (++b1 == L::NB1) b1 = 0;
    if (++cs == L::NC) cs = 0;
  };
  constexpr int UR = L::UR;
  auto renamed = [&](auto phc) -> bool {
    if (!plane(phc)) return false;
    advance();
    return true;
  };
  while (ok && s + UR <= nS) {
    ok = call_in_order(renamed, IntC<0>{}, IntC<UR>{});
    if (!ok) break;
    float4 t[NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) t[i] = a[(i + UR) % NQ];
#pragma unroll
    for (int i = 0; i < NQ; ++i) a[i] = t[i];
  }
  while (ok && s < nS) {
    ok = plane(IntC<0>{});
    if (!ok) break;
    advance();
#pragma unroll
    for (int i = 0; i < 2 * R; ++i) a[i] = a[i + 1];
  }
  if (!ok && lane == 0) {
    *abort_flag = 1;
    atomicExch(p.status, kDevTimeout);
  }
}

}  // namespace dev

// Launch of the two-level pass (radius 4 only).  maps.u: level-n halo box
// (80 x (EY + 2R)); maps.p: extended box (72 x EY) over the field slots;
// maps.cm: extended box of cm.
cudaError_t launch_step2(int R, const StepMaps& maps, const StepParams& p, dim3 grid, cudaStream_t stream) {
  if (R != 4) return cudaErrorInvalidValue;
  using L = dev::Step2Layout<4>;
  static std::atomic<unsigned long long> configured{0};
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (device & 63);
  if (!(configured.load(std::memory_order_acquire) & bit)) {
    e = cudaFuncSetAttribute(dev::step2_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, L::SMEM);
    if (e != cudaSuccess) return e;
    configured.fetch_or(bit, std::memory_order_acq_rel);
  }
  dev::step2_kernel<4><<<grid, L::NTHREADS, L::SMEM, stream>>>(maps.u, maps.p, maps.cm, p);
  return cudaGetLastError();
}

int step2_box(int R, int* ex, int* ey, int* uw, int* uh, int* bx, int* by) {
  if (R != 4) return -1;
  using L = dev::Step2Layout<4>;
  *ex = L::EX;
  *ey = L::EY;
  *uw = L::UW;
  *uh = L::UH;
  *bx = L::BX;
  *by = L::BY;
  return 0;
}

}  // namespace wave
