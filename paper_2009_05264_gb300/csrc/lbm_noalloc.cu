// lbm_step_noalloc: one fused step for callers that cannot allocate device
// memory (code running where cudaMalloc is unavailable or forbidden, such as a
// host that has handed its whole device budget to another allocator, or a
// plug-in inside someone else's memory-managed process).  The caller owns the
// population buffers; the step's scratch -- instance descriptor, step state, tile
// table, fixed-point totals of the partial sums and the diagnostics record -- lives
// in the fixed-size file-scope device array below, which every GPU that loads the
// library holds until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

#include "lbm_internal.h"
#include "pplbm.h"

namespace pplbm {
namespace {

constexpr int kNoAllocMaxTiles = 8192;
constexpr int kNoAllocCols = 128;  // threads per CTA of the fused kernel on this path

// Byte layout of the scratch array (offsets 256-byte aligned).
constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffInst = 0;
constexpr size_t kOffState = align256(kOffInst + sizeof(Inst));
constexpr size_t kOffRing = align256(kOffState + sizeof(InstState));
constexpr size_t kOffSums = align256(kOffRing + sizeof(double) * RING * NDIAG);
constexpr size_t kOffTiles = align256(kOffSums + sizeof(unsigned long long) * 2 * NPART);
constexpr size_t kScratchBytes = align256(kOffTiles + sizeof(Tile) * kNoAllocMaxTiles);

}  // namespace
}  // namespace pplbm

// The scratch of lbm_step_noalloc (about 0.36 MB).  In host code this name is only
// a stand-in for the device array: its device address comes from
// cudaGetSymbolAddress on the current device, at every call, never from taking it
// directly.
static __device__ __align__(256) unsigned char g_lbm_noalloc_scratch[pplbm::kScratchBytes];

namespace pplbm {
namespace {

// Tile table of a (cols - 8)-column, rows-row tiling, written on the device.
__global__ void fill_tiles_kernel(Tile* tiles, int nx, int ny, int w, int rows, int strips, int ntiles) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += gridDim.x * blockDim.x) {
    const int band = t / strips, strip = t - band * strips;
    Tile tl{};
    tl.inst = 0;
    tl.x0 = strip * w;
    tl.y0 = band * rows;
    tl.y1 = min(ny, (band + 1) * rows);
    tl.local = t;
    tl.ntiles = ntiles;
    tiles[t] = tl;
  }
}

// Device address of the scratch array on the current device.  Looked up at every call and
// never kept: a caller's host may reset the device or recreate its primary context between
// calls, which loads the module again at another address.
cudaError_t scratch_on_device(char** out) {
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_lbm_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<char*>(ptr);
  return cudaSuccess;
}

}  // namespace
}  // namespace pplbm

using namespace pplbm;

extern "C" lbm_status lbm_step_noalloc(const lbm_params* p, int32_t nx, int32_t ny, lbm_precision prec,
                                       const void* f_in, const void* g_in, void* f_out, void* g_out,
                                       int32_t in_post_stream, int64_t step, double rho_avg_prev, double* diag_out,
                                       void* cuda_stream) {
  if (nx < 1 || ny < 1 || (prec != LBM_FP32 && prec != LBM_FP64) || step < 0) return LBM_EINVAL;
  if (check_params(nx, ny, p) != nullptr) return LBM_EINVAL;
  if (p->source_model != LBM_SOURCE_GONG_CHENG) return LBM_EINVAL;  // needs a rho^(n-1) history buffer
  if (!f_in || !f_out || f_in == f_out) return LBM_EINVAL;
  if (p->thermal && (!g_in || !g_out || g_in == g_out)) return LBM_EINVAL;
  const long long plane = (long long)nx * ny;
  if (9 * plane >= (1ll << 31)) return LBM_EINVAL;  // 32-bit element offsets in the kernel
  // tiling: 120-column strips; bands tall enough to keep within the scratch's tile table
  const int w = kNoAllocCols - 8;
  const int strips = (nx + w - 1) / w;
  if (strips > kNoAllocMaxTiles) return LBM_EINVAL;
  int rows = default_band_rows(nx, ny, kNoAllocCols, step_wave_slots(prec == LBM_FP64, p->thermal, kNoAllocCols,
                                                                   LBM_KERNEL_SCALAR));
  while ((long long)strips * ((ny + rows - 1) / rows) > kNoAllocMaxTiles) rows *= 2;
  rows = std::min(rows, ny);
  const int ntiles = strips * ((ny + rows - 1) / rows);

  char* base = nullptr;
  if (scratch_on_device(&base) != cudaSuccess) return LBM_ECUDA;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

  Inst I;
  if (fill_inst(I, p, nx, ny, nx, plane, prec == LBM_FP64) != nullptr) return LBM_EINVAL;
  I.rho_prev = nullptr;
  // buffer (step & 1) is read and ((step + 1) & 1) written by the kernel
  I.f[step & 1] = const_cast<void*>(f_in);
  I.f[(step + 1) & 1] = f_out;
  I.g[step & 1] = const_cast<void*>(g_in);
  I.g[(step + 1) & 1] = g_out;
  I.st = reinterpret_cast<InstState*>(base + kOffState);
  I.ring = reinterpret_cast<double*>(base + kOffRing);
  I.sums = reinterpret_cast<unsigned long long*>(base + kOffSums);
  InstState S;
  std::memset(&S, 0, sizeof(S));  // counter and status start at zero on every call
  S.step = step;
  S.local_read = in_post_stream ? 1 : 0;
  S.rho_avg[(step - 1) & 1] = rho_avg_prev;
  S.rho_avg[step & 1] = rho_avg_prev;
  // both copies read host stack memory, staged by the runtime before the calls return
  if (cudaMemcpyAsync(base + kOffInst, &I, sizeof(Inst), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(base + kOffState, &S, sizeof(InstState), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(base + kOffSums, 0, sizeof(unsigned long long) * 2 * NPART, s) != cudaSuccess)
    return LBM_ECUDA;
  Tile* tiles = reinterpret_cast<Tile*>(base + kOffTiles);
  fill_tiles_kernel<<<(ntiles + 255) / 256, 256, 0, s>>>(tiles, nx, ny, w, rows, strips, ntiles);
  if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
  // The caller's buffers are dense (pitch nx, any nx) and only element-aligned, so the
  // paired kernel's 8-byte accesses are not valid here: always the one-column form.
  if (launch_lbm(prec == LBM_FP64, p->thermal, kNoAllocCols, MODE_STEP, LBM_KERNEL_SCALAR, needs_full_step(I),
                 reinterpret_cast<const Inst*>(base + kOffInst), tiles, ntiles, s) != cudaSuccess)
    return LBM_ECUDA;
  InstState out;
  double rec[NDIAG];
  if (cudaMemcpyAsync(&out, base + kOffState, sizeof(InstState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(rec, base + kOffRing + sizeof(double) * (size_t)(step % RING) * NDIAG, sizeof(rec),
                      cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return LBM_ECUDA;
  if (diag_out) std::memcpy(diag_out, rec, sizeof(rec));
  if (out.status & STATUS_BOUNDS) return LBM_EBOUNDS;
  return (out.status & STATUS_UNSTABLE) ? LBM_EUNSTABLE : LBM_OK;
}
