// Internal declarations shared by the CUDA translation units of libwave.
// Not part of the public ABI (see include/wave.h).
#pragma once

#include <cuda.h>            // CUtensorMap type only; the driver is reached through an entry point
#include <cuda_runtime.h>
#include <stdint.h>

namespace wave {

// ---------------------------------------------------------------------------
// Device status word (written by kernels that give up a bounded wait).
// ---------------------------------------------------------------------------
constexpr int kDevOk = 0;
constexpr int kDevTimeout = 1;

// Bounded waits: a kernel gives up after this many nanoseconds of waiting on
// one barrier phase, records kDevTimeout and returns.  This is the default of
// the progress waits (StepParams::wait_ns, settable per context) and the fixed
// limit of the drain waits that let a CTA's issued copies land before it exits.
constexpr unsigned long long kWaitLimitNs = 10ull * 1000ull * 1000ull * 1000ull;

// ---------------------------------------------------------------------------
// Epilogue variants of the stencil step.
// ---------------------------------------------------------------------------
enum StepMode : int {
  MODE_PLAIN = 0,      // new level only (forward, or adjoint without gradient)
  MODE_SNAP_F32 = 1,   // + store the centre level u^n as an FP32 snapshot
  MODE_SNAP_BF16 = 2,  // + BF16 snapshot with per-slab power-of-two scale
  MODE_SNAP_F16 = 3,   // + FP16 snapshot with per-slab power-of-two scale
  MODE_GRAD_F32 = 4,   // adjoint step + imaging condition, FP32 snapshot read
  MODE_GRAD_BF16 = 5,
  MODE_GRAD_F16 = 6,
  MODE_BORN_SRC = 7,   // background step of Born modelling: + writes S = -dm (new - 2 cur + prev)/dt^2
  MODE_SRC = 8,        // step with a source field S added to the Laplacian (scattered field)
  MODE_COUNT = 9
};

__host__ __device__ constexpr bool mode_is_snap(int m) { return m >= MODE_SNAP_F32 && m <= MODE_SNAP_F16; }
__host__ __device__ constexpr bool mode_is_grad(int m) { return m >= MODE_GRAD_F32 && m <= MODE_GRAD_F16; }
// modes that load a third per-point tile through the "g" map (gradient, dm or S)
__host__ __device__ constexpr bool mode_loads_g(int m) { return mode_is_grad(m) || m == MODE_BORN_SRC || m == MODE_SRC; }
// snapshot element format: 0 = f32, 1 = bf16, 2 = f16
__host__ __device__ constexpr int mode_snap_fmt(int m) {
  return m == MODE_SNAP_BF16 || m == MODE_GRAD_BF16 ? 1 : (m == MODE_SNAP_F16 || m == MODE_GRAD_F16 ? 2 : 0);
}

// Snapshot slab for 16-bit storage: 64 points along x by 2 points along axis 1
// of one plane share one power-of-two scale.
constexpr int kSlabX = 64;
constexpr int kSlabY = 2;

// ---------------------------------------------------------------------------
// Tile geometry of the stencil step, per stencil radius R and dimension.
// A CTA owns BX x BY output columns (x, axis 1) and streams a chunk of planes
// along axis 2 (3D); in 2D it owns one BX x BY tile of the single plane.
// ---------------------------------------------------------------------------
// Radius from which the lead-plane design is used (every mode).
constexpr int kLeadMinR = 7;
// Radius from which equal spacing on every axis selects the kernel variant
// with one coefficient per offset (with 14-row tiles at 128 registers: order 12
// forward step 0.645 -> 0.579 ms on 592^3; order 14 and 16 likewise faster).
constexpr int kIsoMinR = 6;
__host__ __device__ constexpr bool iso_kernel(int R, bool equal_spacing) { return equal_spacing && R >= kIsoMinR; }
// Planes per renamed register-queue group where a full period of 2R+1 planes
// would spill (see StepLayout::UR).
constexpr int kRenameGroup = 4;

// Shared memory of one SM and the part the driver keeps per resident CTA.
constexpr int kSmemPerSm = 228 * 1024;
constexpr int kSmemReservedPerCta = 1024;
constexpr int kSmemTwoCtas = kSmemPerSm / 2 - kSmemReservedPerCta;  // per CTA at two CTAs per SM

template <int R, int NDIM, bool ISO = false>
struct StepTraits {
  static constexpr int BX = 64;                   // x outputs per CTA (16 threads x 4)
  // axis-1 outputs per CTA (one row per 16 threads, two rows per warp); 3D
  // radius 8, and radius 6-7 with the equal-spacing kernel, use 14 rows so
  // that a CTA has 8 warps and two CTAs fit the register file at 128 registers
  // per thread (measured slower for the general radius-7 kernel; the order-12
  // equal-spacing step 0.594 -> 0.579 ms against 16 rows at 96 registers)
  static constexpr int BY = (NDIM == 3 && (R >= 8 || (R >= 6 && ISO))) ? 14 : 16;
  static constexpr int HX = (R <= 4) ? 4 : 8;     // x halo, rounded to 16 bytes for TMA
  static constexpr int RZ = (NDIM == 3) ? R : 0;  // halo along the streamed axis
  static constexpr int UW = BX + 2 * HX;          // smem row length of a halo box (floats)
  static constexpr int UH = BY + 2 * R;           // rows of a halo box
  static constexpr int U_BYTES = UW * UH * 4;                // bytes of one halo box
  static constexpr int U_STRIDE = (U_BYTES + 127) / 128 * 128;  // halo box spacing (128-byte aligned)
  static constexpr int T_ELEMS = BX * BY;
  static constexpr int NCW = BY / 2;              // consumer warps
  static constexpr int NTHREADS = (NCW + 1) * 32; // + one producer warp
};

// Shared-memory layout, prefetch depth and occupancy of one (R, NDIM, MODE, ISO).
template <int R, int NDIM, int MODE, bool ISO = false>
struct StepLayout {
  using T = StepTraits<R, NDIM, ISO>;
  static constexpr int HX = T::HX;
  static constexpr int RZ = T::RZ;
  static constexpr int SNAP_ELEM = mode_snap_fmt(MODE) == 0 ? 4 : 2;
  // per-point tiles loaded with each plane: previous level, cm, and g (the
  // gradient, dm or S) and the snapshot where the mode needs them
  static constexpr int TILE_BYTES = mode_is_grad(MODE) ? (3 * T::T_ELEMS * 4 + T::T_ELEMS * SNAP_ELEM)
                                                       : (mode_loads_g(MODE) ? 3 : 2) * T::T_ELEMS * 4;
  // Shared memory of a layout: `lead` selects the design, pf planes are
  // prefetched ahead, nsp stages hold the per-point tiles.
  //  * classic: the queue-feed ring holds halo planes z .. z+R+pf;
  //  * lead-plane: the register queue is fed from a small ring of interior
  //    boxes of plane z+R, and the halo box of the centre plane is loaded again
  //    (from L2) with the per-point tiles, so the shared ring holds only the
  //    prefetch depth instead of R+1+pf halo planes.
  static constexpr int nsu_of(bool lead, int pf) { return lead ? pf + 1 : T::RZ + 1 + pf; }
  static constexpr int qstride_of(bool lead) { return lead ? T::T_ELEMS * 4 : T::U_STRIDE; }
  static constexpr int pbytes_of(bool lead) { return (lead ? T::U_STRIDE : 0) + TILE_BYTES; }
  // 2*(NSU+NSP) mbarriers + an abort flag, padded to 128 bytes
  static constexpr int bar_bytes(int nsu, int nsp) { return ((16 * (nsu + nsp) + 16 + 127) / 128) * 128; }
  static constexpr int smem_of(bool lead, int pf, int nsp) {
    return bar_bytes(nsu_of(lead, pf), nsp) + nsu_of(lead, pf) * qstride_of(lead) + nsp * pbytes_of(lead) + 128;
  }
  static constexpr bool fits(bool lead, int pf, int nsp) { return smem_of(lead, pf, nsp) <= kSmemTwoCtas; }

  // Lead-plane design from radius 7 on for every step; from radius 3 for the
  // plain and 16-bit-snapshot steps and from radius 5 for the FP32-snapshot
  // and 16-bit imaging steps, where it was measured faster on 592^3 (order 8
  // plain step 0.530 -> 0.519 ms, order 10 FP32 snapshot 0.663 -> 0.647 ms,
  // order 10 FP16 imaging 0.886 -> 0.847 ms; the FP32 snapshot and imaging
  // steps up to radius 4 were slower: 0.640 -> 0.658 and 0.854 -> 0.883 ms at
  // order 8); and wherever the classic design would not fit two CTAs per SM.
  static constexpr bool LEAD_PREFERRED =
      R >= kLeadMinR ||
      (R >= 3 && (MODE == MODE_PLAIN || MODE == MODE_SNAP_BF16 || MODE == MODE_SNAP_F16)) ||
      (R >= 5 && (MODE == MODE_SNAP_F32 || MODE == MODE_GRAD_BF16 || MODE == MODE_GRAD_F16));
  static constexpr bool LEAD = (NDIM == 3) && (LEAD_PREFERRED || !fits(false, 2, 3));
  // Deep variant (classic design, not the imaging condition): two CTAs per SM
  // with a 4-plane prefetch (3 where 4 would not fit two CTAs) and, up to
  // radius 2, output planes taken in pairs (half the register-queue moves),
  // which the 96 registers per thread at two CTAs allow.
  static constexpr int DEEP_PF = fits(false, 4, 3) ? 4 : (fits(false, 3, 3) ? 3 : 0);
  static constexpr bool DEEP = NDIM == 3 && !LEAD && !mode_is_grad(MODE) && DEEP_PF > 0;
  // The imaging steps are HBM-bound and keep a 2-plane prefetch; with 16-bit
  // snapshots their per-plane stages are smaller, and a 3-plane prefetch with
  // a 4-stage per-point ring keeps more bytes in flight where it fits.
  static constexpr bool G16_DEEP =
      NDIM == 3 && mode_is_grad(MODE) && mode_snap_fmt(MODE) != 0 && fits(LEAD, 3, 4);
  // Lead-plane kernels from radius 7 (every mode): the deepest prefetch of 4
  // planes (5 per-point stages) or 3 (4 stages) that fits two CTAs per SM.
  // Their register queue and per-plane arithmetic leave the ring little slack:
  // order 16 forward 0.838 -> 0.827 ms, snapshot 0.884 -> 0.860 ms, FP32
  // imaging 0.982 -> 0.964 ms on 592^3.
  static constexpr int LEAD_PF =
      (NDIM == 3 && LEAD && LEAD_PREFERRED) ? (fits(true, 4, 5) ? 4 : (fits(true, 3, 4) ? 3 : 0)) : 0;
  static constexpr int PF =
      NDIM == 3 ? (DEEP ? DEEP_PF : (LEAD_PF > 0 ? LEAD_PF : (G16_DEEP ? 3 : 2))) : 0;  // planes prefetched ahead
  static constexpr int NSP =
      NDIM == 3 ? (LEAD_PF > 0 ? LEAD_PF + 1 : (G16_DEEP ? 4 : 3)) : 1;  // per-point ring stages
  static constexpr int NSU = nsu_of(LEAD, PF);                                       // queue-feed ring stages
  static constexpr int Q_BYTES = LEAD ? T::T_ELEMS * 4 : T::U_BYTES;
  static constexpr int Q_STRIDE = qstride_of(LEAD);
  static constexpr int QU = (DEEP && R <= 2) ? 2 : 1;  // output planes per register-queue move
  // Output planes per renamed group (1 = the queue moves after every plane):
  // the 2R+1 queue slots are renamed over a group of UR planes and rotated
  // once after it (2R+2 moves per group instead of 2R per plane); a group of
  // a full period, 2R+1 planes, needs no rotation at all.  Chosen per kernel
  // from measurements on 592^3 and the ptxas spill counts:
  //  * full period for the deep forward / snapshot steps at radius 3-4 and the
  //    FP32 imaging step at radius 4 (order 8 forward 0.545 -> 0.524 ms);
  //  * groups of 4 for the other kernels up to radius 6 (order 12 forward
  //    0.710 -> 0.667 ms, 16-bit imaging steps 4-6 % faster) and the
  //    equal-spacing kernels from radius 7 (order 16 forward 0.934 -> 0.837 ms);
  //  * none where a group spills under the register cap (imaging at radius 5,
  //    16-bit snapshot, imaging and Born steps at radius 6 with general
  //    spacing, general spacing from radius 7) and for the paired planes of
  //    the deep steps up to radius 2 (no measurable difference there); the
  //    equal-spacing radius-6 kernels, at 128 registers, take groups (order 12
  //    FP16 snapshot step 0.722 -> 0.658 ms, FP16 imaging 0.871 -> 0.850 ms).
  static constexpr int UR_BASE =
      (NDIM != 3 || QU != 1) ? 1
      : (R >= kLeadMinR) ? (ISO ? kRenameGroup : 1)
      : ((R == 5 && mode_is_grad(MODE)) || (R == 6 && MODE >= MODE_SNAP_BF16 && !ISO)) ? 1
      : ((DEEP && (R == 3 || R == 4)) || (R == 4 && MODE == MODE_GRAD_F32)) ? 2 * R + 1
      : kRenameGroup;
  // Lead-plane layouts take one stage per plane for both rings: stage s holds
  // the queue box of plane z0 - RZ + s and, from s = 2RZ on, the per-point
  // tiles of plane s - 2RZ, under one full and one empty barrier (one wait and
  // one release per plane).  Their renamed groups span exactly the NSU stages,
  // so that within a group every stage slot is a compile-time offset and the
  // phase flips once per group.
  static constexpr bool COMBINED = LEAD;
  // One-ring kernels: the consumers load the first 2RZ queue planes of a
  // column run themselves (independent 16-byte loads, all in flight) instead
  // of taking them through the ring a few stages at a time; the ring starts at
  // output plane 0.
  static constexpr bool DIRECT_FILL = COMBINED;
  static constexpr int UR = (COMBINED && UR_BASE > 1) ? nsu_of(LEAD, PF) : UR_BASE;
  // Damped points on packed pairs (the same values as one point at a time)
  // where measured faster on 592^3: the FP32 snapshot steps up to radius 4
  // (order 8 0.640 -> 0.632 ms) and the 16-bit snapshot steps at radius 8
  // (order 16 FP16 0.822 -> 0.795 ms); elsewhere the extra live pairs cost
  // more than the halved arithmetic (order 16 forward 0.708 -> 0.728 ms).
  static constexpr bool PACKED_DAMP =
      (MODE == MODE_SNAP_F32 && R <= 4) || ((MODE == MODE_SNAP_BF16 || MODE == MODE_SNAP_F16) && R == 8);
  // resident CTAs per SM asked of the register allocator (registers per
  // thread follow the warps per SM sub-partition: 3 CTAs of 9 warps leave 72,
  // 2 of 9 leave 96, 2 of 8 leave 128)
  static constexpr int MIN_BLOCKS = (NDIM == 2 && R <= 4 && !mode_is_grad(MODE)) ? 3 : 2;

  static constexpr int HALO_OFF = 0;                        // lead design: centre halo box
  static constexpr int PREV_OFF = LEAD ? T::U_STRIDE : 0;
  static constexpr int CM_OFF = PREV_OFF + T::T_ELEMS * 4;
  static constexpr int G_OFF = CM_OFF + T::T_ELEMS * 4;
  static constexpr int S_OFF = G_OFF + T::T_ELEMS * 4;
  static constexpr int P_TX = (LEAD ? T::U_BYTES : 0) + TILE_BYTES;  // bytes landing per plane stage
  static constexpr int P_BYTES = pbytes_of(LEAD);                      // stage spacing
  static_assert(P_BYTES % 128 == 0, "per-point stage must keep 128-byte alignment");
  static constexpr int BAR_BYTES = bar_bytes(NSU, NSP);
  static constexpr int U_OFF = BAR_BYTES;
  static constexpr int PST_OFF = U_OFF + NSU * Q_STRIDE;
  static constexpr int SMEM = PST_OFF + NSP * P_BYTES + 128;  // + runtime 128-byte alignment
};

// ---------------------------------------------------------------------------
// Launch parameters of one stencil step (one time level).
// Field buffer: 4 wavefield slots [slot][NZ][NY][pitch] float32.
// ---------------------------------------------------------------------------
struct StepParams {
  int NX, NY, NZ;          // computational points per kernel axis
  int pitch;               // floats per row (multiple of 8)
  int zchunk;              // planes per CTA along axis 2
  int cur, prev;           // field slots: centre level and previous level (overwritten by the new level)
  float* fields;           // base of the field buffer
  long long slot_elems;    // elements per field slot (NZ*NY*pitch)
  // stencil coefficients (1/h^2 folded in): lap = c0*u + sum_j c{x,y,z}[j-1]*(u[-j]+u[+j])
  float c0;
  float cx[8], cy[8], cz[8];
  int iso;                 // 1: equal-spacing kernel variant (cx == cy (== cz), radius >= kIsoMinR)
  // sponge: eta = sum_axis eta_max_axis * (delta/nbl)^2 ; nbl per kernel axis (0 on a missing axis)
  int nblx, nbly, nblz;
  float emx, emy, emz;     // eta_max per axis divided by nbl^2 (1/ms)
  float half_inv_dt;       // 0.5/dt
  float inv_dt2;           // 1/dt^2
  // snapshot store (SNAP modes): level base pointer and slab scales
  void* snap_out;
  float* scale_out;
  // gradient (GRAD modes) or Born source field written by MODE_BORN_SRC
  float* grad;             // [NZ][NY][pitch]
  int snap_level;          // level coordinate in the snapshot store
  const float* scale_in;   // slab scales of that level
  int slabs_x, slabs_y;    // slab grid per plane
  int* status;             // device status word
  unsigned long long wait_ns;  // limit of each progress wait (the drain waits keep kWaitLimitNs)
  int withhold;            // test hook: 1 = the producer issues no tile loads (every consumer wait runs out)
  int out1, out2;          // two-level pass: field slots receiving levels n+1 and n+2
};

// Host-side launcher for one (R, NDIM, MODE); defined in step_r<R>.cu.
struct StepMaps {
  CUtensorMap u;   // field buffer, halo box  (4D: x, y, z, slot)
  CUtensorMap p;   // field buffer, tile box  (4D)
  CUtensorMap cm;  // coefficient dt^2/m, tile box (3D)
  CUtensorMap g;   // gradient, tile box (3D)
  CUtensorMap s;   // snapshot store, tile box (4D: x, y, z, level)
};

// One resident request of a batched step launch (serving): the CTAs
// [cta0, cta0 + tiles_x * tiles_y * chunks) of the launch run the request's
// step n0 + k (k: the launch's index within the call) while n0 + k < nlast.
// Lives in device memory; the tensor maps are read from there.
struct alignas(64) BatchStep {
  StepMaps maps;
  StepParams p;
  int cta0;
  int tiles_x, tiles_y;
  int n0, nlast;
};
// Launches the step kernel variant of p.iso.
cudaError_t launch_step(int R, int ndim, int mode, const StepMaps& maps, const StepParams& p,
                        dim3 grid, cudaStream_t stream);
// Two-level pass (step2_kernel.cu): levels n+1 and n+2 of a source-free 3D
// forward step pair at radius 4 from slots p.prev (n-1) and p.cur (n) into
// p.out1 and p.out2, which must differ from both.  step2_box gives its tile
// geometry (extended tile, level-n halo box, output tile); -1 where the pass
// does not exist.
cudaError_t launch_step2(int R, const StepMaps& maps, const StepParams& p, dim3 grid, cudaStream_t stream);
int step2_box(int R, int* ex, int* ey, int* uw, int* uh, int* bx, int* by);
// Batched plain step of nreq requests sharing (R, ndim, iso): `ctas` CTAs in
// all, table in device memory; launch index k within the call.
cudaError_t launch_step_batch(int R, int ndim, bool iso, const BatchStep* table, int nreq, int ctas, int k,
                              cudaStream_t stream);
// Tile geometry of StepTraits<R, NDIM, iso> for the host (maps and grid).
int step_smem_bytes(int R, int ndim, int mode, bool iso);
// Compile-time configuration of the step kernel launched for (R, ndim, mode,
// equal spacing); returns the number of values written to out (at most
// kStepLayoutMax).
constexpr int kStepLayoutMax = 32;
int step_layout(int R, int ndim, int mode, bool iso, int* out);
int step_bx();
int step_by(int R, int ndim, bool iso);
int step_hx(int R);

// ---------------------------------------------------------------------------
// Auxiliary kernels (aux_kernels.cu)
// ---------------------------------------------------------------------------
struct GridDims {
  int NX, NY, NZ, pitch;
  int nblx, nbly, nblz;    // sponge width per kernel axis
  int PX, PY, PZ;          // physical points per kernel axis
};

cudaError_t launch_setup_cm(const GridDims& g, const float* m_phys, float* cm, float dt2, cudaStream_t s);
cudaError_t launch_minmax(const float* m, long long n, unsigned int* out_minmax_bits, cudaStream_t s);

// sparse points: gather (receiver sampling) and CSR injection
struct GatherSet {
  long long n;             // points
  const long long* base;   // linear index of corner (0,0,0)
  const float* frac;       // [n][3] fractions (x, axis1, axis2)
  int ndim;
  long long sy, sz;        // linear strides of axis 1 and axis 2
};
struct InjectSet {
  int n;                   // unique grid cells
  const long long* cell;   // linear index per cell
  const int* rowptr;       // [n+1]
  const int* pidx;         // contributing point per entry
  const float* w;          // weight per entry
  float* coef;             // per cell cm/(1+k), filled by launch_inject_coef
};
// Source injection and receiver sampling of one request in a batched launch
// (step n = n0 + k: injection of row n into level n+1, gather of row n+1).
struct BatchSparse {
  InjectSet inj;
  const float* q;          // [nt][ns]
  long long ns;
  GatherSet gat;
  float* d;                // [nt][nr]
  float* fields;           // the request's two field slots
  long long slot_elems;
  int n0, nlast;
  int gcta0;               // first CTA of the request's gather in the launch
};

// Column segments of the plain 3D step, for grids of few CTA waves: the
// tiles_x * tiles_y columns of NZ planes, tile after tile, form one sequence
// of planes, cut into one run per CTA, [run_start[b], run_start[b+1]) for CTA
// b (a run may end in one column and go on at the top of the next).  Such a
// launch also does the step's sparse work: the injection of source row n into
// the cells of the CTA's runs once its planes are written (inj_vals = row n,
// or null), and the sampling of receiver row n from the centre level, a share
// of the receivers per CTA, while its first planes load (rec_out = row n, or
// null).
struct SegWork {
  const long long* run_start;  // [ctas + 1], device
  int tiles_x, tiles_y;
  InjectSet inj;
  const int* inj_ptr;      // [ctas + 1]: the CTA's cells in inj_list
  const int* inj_list;     // indices into inj, grouped by CTA
  const float* inj_vals;   // source row n, or null
  GatherSet rec;
  float* rec_out;          // receiver row n, or null
};
// Segmented plain step (3D) of `ctas` CTAs; the variant of p.iso.
cudaError_t launch_step_seg(int R, bool iso, const StepMaps& maps, const StepParams& p, const SegWork& w, int ctas,
                            cudaStream_t stream);

cudaError_t launch_gather(const GatherSet& gs, const float* field, float* out_row, cudaStream_t s);
cudaError_t launch_inject_coef(const InjectSet& is, const GridDims& g, const float* cm,
                               const float* eta_max_over_nbl2, float half_inv_dt, cudaStream_t s);
cudaError_t launch_inject(const InjectSet& is, const float* values_row, float* field, cudaStream_t s);
// injection during the gradient sweep: also corrects the imaging condition at the cell
cudaError_t launch_inject_grad(const InjectSet& is, const float* values_row, float* field, float* grad,
                               const void* snap_level, int snap_fmt, const float* scale_level,
                               const GridDims& g, int slabs_x, int slabs_y, float inv_dt2, cudaStream_t s);

cudaError_t launch_residual(const float* d, const float* d_obs, float* r, long long n,
                            double* partials, int nblocks, cudaStream_t s);
cudaError_t launch_sum_partials(const double* partials, int n, double* out, cudaStream_t s);
int residual_blocks(long long n);

cudaError_t launch_fold(const GridDims& g, const float* grad_comp, float* grad_phys, cudaStream_t s);
cudaError_t launch_snapshot_store(const GridDims& g, const float* field, void* snap, float* scale,
                                  int fmt, int slabs_x, int slabs_y, cudaStream_t s);
cudaError_t launch_pack_state(const GridDims& g, const float* field, float* dense, cudaStream_t s);
cudaError_t launch_unpack_state(const GridDims& g, const float* dense, float* field, cudaStream_t s);
cudaError_t launch_fill_zero(float* p, long long n, cudaStream_t s);
// physical field -> computational grid by edge replication (pitched, zero padding columns)
cudaError_t launch_pad_field(const GridDims& g, const float* phys, float* comp, cudaStream_t s);
// graph-replay variants: time row = *counter + offset (+1 for the gather)
cudaError_t launch_inject_counter(const InjectSet& is, const float* q, long long ns, const int* counter, int offset,
                                  float* field, cudaStream_t s);
cudaError_t launch_gather_counter(const GatherSet& gs, const float* field, float* d, const int* counter, int offset,
                                  cudaStream_t s);
cudaError_t launch_counter_add(int* counter, int delta, cudaStream_t s);
// batched injection (one CTA per request) and receiver sampling (gather CTAs
// of the requests one after another, gather_ctas in all) of launch index k
cudaError_t launch_inject_batch(const BatchSparse* table, int nreq, int k, cudaStream_t s);
cudaError_t launch_gather_batch(const BatchSparse* table, int nreq, int gather_ctas, int k, cudaStream_t s);
int gather_batch_ctas(long long npoints, int ndim);

}  // namespace wave
