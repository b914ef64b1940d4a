// Kernel instantiations for double storage and arithmetic.
#include "lbm_kernels.cuh"

namespace pplbm {

cudaError_t launch_lbm_f64(int thermal, int cols, int mode, int kernel, bool full, const Inst* d_inst,
                          const Tile* d_tiles, int ntiles, cudaStream_t s, const Inst* h_inst) {
  return launch_precision<double>(thermal, cols, mode, full, mode == MODE_STEP && kernel == LBM_KERNEL_INTERIOR, d_inst,
                                  d_tiles, ntiles, s, h_inst);
}

cudaError_t launch_persistent_f64(int thermal, int cols, int kernel, bool full, const Inst* d_inst,
                                  const Tile* d_tiles, int ntiles, int nsteps, GridBar* bar, unsigned max_polls,
                                  cudaStream_t s, const Inst* h_inst, const FlowPlan& flow) {
  return launch_persistent_precision<double>(thermal, cols, full, kernel == LBM_KERNEL_INTERIOR, d_inst, d_tiles,
                                             ntiles, nsteps, bar, max_polls, s, h_inst, flow);
}

int persistent_resident_f64(int thermal, int cols, int kernel, bool full, bool single) {
  return persistent_resident_precision<double>(thermal, cols, full, kernel == LBM_KERNEL_INTERIOR, single);
}

int resident_ctas_f64(int thermal, int cols, int kernel) {
  return resident_precision<double>(thermal, cols, kernel == LBM_KERNEL_INTERIOR);
}

cudaError_t launch_init_from_fields_f64(const Inst* d_inst, int nx, int ny, const double* d_fields, int has_T,
                                       cudaStream_t s) {
  return launch_init_fields_t<double>(d_inst, nx, ny, d_fields, has_T, s);
}

cudaError_t launch_init_builtin_f64(const Inst* d_inst, int nx, int ny, InitSpec spec, cudaStream_t s) {
  return launch_init_builtin_t<double>(d_inst, nx, ny, spec, s);
}

}  // namespace pplbm
