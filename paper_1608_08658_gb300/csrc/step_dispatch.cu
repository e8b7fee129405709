// Runtime dispatch of the stencil step over the stencil radius.
#include "step_launch.cuh"

namespace wave {

#define WAVE_DECLARE_RADIUS(RR)                                                                          \
  cudaError_t launch_step_r##RR(int ndim, int mode, const StepMaps& maps, const StepParams& p, dim3 grid, \
                                cudaStream_t s);                                                        \
  int step_smem_r##RR(int ndim, int mode, bool iso);                                                    \
  int step_layout_r##RR(int ndim, int mode, bool iso, int* out);                                        \
  cudaError_t launch_step_batch_r##RR(int ndim, bool iso, const BatchStep* table, int nreq, int ctas, int k,     \
                                      cudaStream_t s);                                                  \
  cudaError_t launch_step_seg_r##RR(bool iso, const StepMaps& maps, const StepParams& p, const SegWork& w, int ctas, \
                                    cudaStream_t s);
WAVE_DECLARE_RADIUS(1)
WAVE_DECLARE_RADIUS(2)
WAVE_DECLARE_RADIUS(3)
WAVE_DECLARE_RADIUS(4)
WAVE_DECLARE_RADIUS(5)
WAVE_DECLARE_RADIUS(6)
WAVE_DECLARE_RADIUS(7)
WAVE_DECLARE_RADIUS(8)

cudaError_t launch_step(int R, int ndim, int mode, const StepMaps& maps, const StepParams& p, dim3 grid,
                        cudaStream_t stream) {
  switch (R) {
    case 1: return launch_step_r1(ndim, mode, maps, p, grid, stream);
    case 2: return launch_step_r2(ndim, mode, maps, p, grid, stream);
    case 3: return launch_step_r3(ndim, mode, maps, p, grid, stream);
    case 4: return launch_step_r4(ndim, mode, maps, p, grid, stream);
    case 5: return launch_step_r5(ndim, mode, maps, p, grid, stream);
    case 6: return launch_step_r6(ndim, mode, maps, p, grid, stream);
    case 7: return launch_step_r7(ndim, mode, maps, p, grid, stream);
    case 8: return launch_step_r8(ndim, mode, maps, p, grid, stream);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_step_batch(int R, int ndim, bool iso, const BatchStep* table, int nreq, int ctas, int k,
                              cudaStream_t s) {
  switch (R) {
    case 1: return launch_step_batch_r1(ndim, iso, table, nreq, ctas, k, s);
    case 2: return launch_step_batch_r2(ndim, iso, table, nreq, ctas, k, s);
    case 3: return launch_step_batch_r3(ndim, iso, table, nreq, ctas, k, s);
    case 4: return launch_step_batch_r4(ndim, iso, table, nreq, ctas, k, s);
    case 5: return launch_step_batch_r5(ndim, iso, table, nreq, ctas, k, s);
    case 6: return launch_step_batch_r6(ndim, iso, table, nreq, ctas, k, s);
    case 7: return launch_step_batch_r7(ndim, iso, table, nreq, ctas, k, s);
    case 8: return launch_step_batch_r8(ndim, iso, table, nreq, ctas, k, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_step_seg(int R, bool iso, const StepMaps& maps, const StepParams& p, const SegWork& w, int ctas,
                            cudaStream_t s) {
  switch (R) {
    case 1: return launch_step_seg_r1(iso, maps, p, w, ctas, s);
    case 2: return launch_step_seg_r2(iso, maps, p, w, ctas, s);
    case 3: return launch_step_seg_r3(iso, maps, p, w, ctas, s);
    case 4: return launch_step_seg_r4(iso, maps, p, w, ctas, s);
    case 5: return launch_step_seg_r5(iso, maps, p, w, ctas, s);
    case 6: return launch_step_seg_r6(iso, maps, p, w, ctas, s);
    case 7: return launch_step_seg_r7(iso, maps, p, w, ctas, s);
    case 8: return launch_step_seg_r8(iso, maps, p, w, ctas, s);
    default: return cudaErrorInvalidValue;
  }
}

int step_smem_bytes(int R, int ndim, int mode, bool iso) {
  switch (R) {
    case 1: return step_smem_r1(ndim, mode, iso);
    case 2: return step_smem_r2(ndim, mode, iso);
    case 3: return step_smem_r3(ndim, mode, iso);
    case 4: return step_smem_r4(ndim, mode, iso);
    case 5: return step_smem_r5(ndim, mode, iso);
    case 6: return step_smem_r6(ndim, mode, iso);
    case 7: return step_smem_r7(ndim, mode, iso);
    case 8: return step_smem_r8(ndim, mode, iso);
    default: return -1;
  }
}

int step_layout(int R, int ndim, int mode, bool iso, int* out) {
  switch (R) {
    case 1: return step_layout_r1(ndim, mode, iso, out);
    case 2: return step_layout_r2(ndim, mode, iso, out);
    case 3: return step_layout_r3(ndim, mode, iso, out);
    case 4: return step_layout_r4(ndim, mode, iso, out);
    case 5: return step_layout_r5(ndim, mode, iso, out);
    case 6: return step_layout_r6(ndim, mode, iso, out);
    case 7: return step_layout_r7(ndim, mode, iso, out);
    case 8: return step_layout_r8(ndim, mode, iso, out);
    default: return -1;
  }
}

int step_bx() { return StepTraits<1, 3>::BX; }
int step_by(int R, int ndim, bool iso) {
  if (ndim != 3) return StepTraits<1, 2>::BY;
  if (iso_kernel(R, iso)) {
    switch (R) {
      case 6: return StepTraits<6, 3, true>::BY;
      case 7: return StepTraits<7, 3, true>::BY;
      default: return StepTraits<8, 3, true>::BY;
    }
  }
  switch (R) {
    case 1: return StepTraits<1, 3>::BY;
    case 2: return StepTraits<2, 3>::BY;
    case 3: return StepTraits<3, 3>::BY;
    case 4: return StepTraits<4, 3>::BY;
    case 5: return StepTraits<5, 3>::BY;
    case 6: return StepTraits<6, 3>::BY;
    case 7: return StepTraits<7, 3>::BY;
    case 8: return StepTraits<8, 3>::BY;
    default: return -1;
  }
}
int step_hx(int R) { return R <= 4 ? 4 : 8; }

}  // namespace wave
