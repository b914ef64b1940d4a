// Kernel instantiations for float storage and arithmetic.
#include "lbm_kernels.cuh"
#include "lbm_pair.cuh"
#include "lbm_tma.cuh"

namespace pplbm {

cudaError_t launch_lbm_f32(int thermal, int cols, int mode, int kernel, bool full, const Inst* d_inst,
                          const Tile* d_tiles, int ntiles, cudaStream_t s, const Inst* h_inst, unsigned max_polls) {
  if (mode == MODE_STEP && kernel == LBM_KERNEL_PAIRED) return launch_pair(thermal, cols, d_inst, d_tiles, ntiles, s);
  if (mode == MODE_STEP && kernel == LBM_KERNEL_TMA)
    return launch_tma(thermal, cols, d_inst, d_tiles, ntiles, s, h_inst, max_polls);
  return launch_precision<float>(thermal, cols, mode, full, mode == MODE_STEP && kernel == LBM_KERNEL_INTERIOR, d_inst,
                                 d_tiles, ntiles, s, h_inst);
}

cudaError_t launch_persistent_f32(int thermal, int cols, int kernel, bool full, const Inst* d_inst,
                                  const Tile* d_tiles, int ntiles, int nsteps, GridBar* bar, unsigned max_polls,
                                  cudaStream_t s, const Inst* h_inst, const FlowPlan& flow) {
  if (kernel != LBM_KERNEL_SCALAR && kernel != LBM_KERNEL_INTERIOR) return cudaErrorNotSupported;
  return launch_persistent_precision<float>(thermal, cols, full, kernel == LBM_KERNEL_INTERIOR, d_inst, d_tiles,
                                            ntiles, nsteps, bar, max_polls, s, h_inst, flow);
}

int persistent_resident_f32(int thermal, int cols, int kernel, bool full, bool single) {
  return persistent_resident_precision<float>(thermal, cols, full, kernel == LBM_KERNEL_INTERIOR, single);
}

int resident_ctas_f32(int thermal, int cols, int kernel) {
  if (kernel == LBM_KERNEL_PAIRED) return resident_pair(thermal, cols);
  if (kernel == LBM_KERNEL_TMA && cols == ST_COLS) return resident_tma(thermal);
  return resident_precision<float>(thermal, cols, kernel == LBM_KERNEL_INTERIOR);
}

cudaError_t launch_init_from_fields_f32(const Inst* d_inst, int nx, int ny, const double* d_fields, int has_T,
                                       cudaStream_t s) {
  return launch_init_fields_t<float>(d_inst, nx, ny, d_fields, has_T, s);
}

cudaError_t launch_init_builtin_f32(const Inst* d_inst, int nx, int ny, InitSpec spec, cudaStream_t s) {
  return launch_init_builtin_t<float>(d_inst, nx, ny, spec, s);
}

}  // namespace pplbm
