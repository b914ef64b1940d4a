// Batches of independent lattices advanced by one fused launch per step.
//
// A batch owns member contexts (each with its own populations, step state,
// partial sums and diagnostics ring, created on the batch's stream) and a
// concatenated tile table over all members; one launch of the fused kernel per
// step covers every member's tiles, so lattices of uneven size and parameters
// share the GPU in one grid.  Each member's partials go into that member's own
// totals, taken by its last tile, so per-member results are those of the member run
// alone with the same tiling.  Runs of steps are captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm_internal.h"
#include "pplbm.h"

using namespace pplbm;

namespace {

constexpr int kGraphChunk = 16;  // steps per captured graph

struct Member {
  lbm_ctx* ctx = nullptr;
  int nx = 0, ny = 0;
  unsigned long long gen = 0;  // descriptor generation copied into the device table
};

}  // namespace

struct lbm_batch {
  lbm_precision prec = LBM_FP32;
  int thermal = 1;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<Member> slots;  // empty ctx = free slot
  int cols = 128, rows = 0;   // rows 0: each member's default band height
  int kernel = LBM_KERNEL_AUTO;         // requested step kernel form
  int launch_kernel = LBM_KERNEL_SCALAR; // the form the batch's launches take (resolve_kernel)
  bool any_full = false;  // a member needs the step's full form (pool, Hazi-Markus, bubble statistics)
  // device tables of the current membership
  Inst* d_insts = nullptr;
  Tile* d_tiles = nullptr;
  size_t cap_insts = 0, cap_tiles = 0;
  int ntiles = 0;
  bool dirty = true;
  cudaGraphExec_t graph = nullptr;
  long long launches = 0;
  int loop = LBM_LOOP_AUTO;     // requested step loop
  unsigned max_polls = 0;        // barrier polls before a persistent launch gives up (0: time limit only)
  GridBar* d_bar = nullptr;      // grid barrier of the persistent launches (allocated on first use)
  // overlapped persistent launches: per member its tiling, its step at the launch's start, and
  // per tile position the steps finished (capacities follow the descriptor and tile tables)
  FlowInst* d_flow = nullptr;
  long long* d_step0 = nullptr;
  unsigned long long* d_cells = nullptr;
  bool flow_ok = false;  // every member may run overlapped (no pool, distinct inlet and outlet)
  std::string err;
};

namespace {

lbm_status bfail(lbm_batch* b, lbm_status s, const std::string& msg) {
  if (b) b->err = msg;
  return s;
}

#define LBM_BCUDA(b, call)                                                                     \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return bfail(b, LBM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

void drop_graph(lbm_batch* b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
}

// Band plan of a member: uniform bands of the batch's explicit height, or the default plan
// for the member's share of one wave's CTA slots (in proportion to its share of the batch's
// nodes).
BandPlan member_plan(const lbm_batch* b, int nx, int ny, long long slots, double share) {
  if (b->rows > 0) return BandPlan{0, 0, std::max(1, std::min(b->rows, ny))};
  const long long member_slots = std::max<long long>(1, (long long)(slots * share + 0.5));
  return default_band_plan(nx, ny, b->cols, member_slots);
}

// Upload the descriptors and the concatenated tile table of the active members.
lbm_status rebuild(lbm_batch* b) {
  std::vector<Inst> insts;
  std::vector<Tile> tiles;
  bool any_hazi = false;  // a member uses the Hazi-Markus source (no paired form)
  bool any_full = false;
  bool all_tmaps = true;  // every member has the tensor maps of the TMA kernel
  const int w = b->cols - 8;
  double total = 0.0;
  for (const Member& m : b->slots) {
    if (!m.ctx) continue;
    total += (double)m.nx * m.ny;
    const Inst I = lbm_internal_inst(m.ctx);
    any_hazi = any_hazi || I.source_model == LBM_SOURCE_HAZI_MARKUS;
    any_full = any_full || needs_full_step(I);
    all_tmaps = all_tmaps && I.tmaps != nullptr;
  }
  const int launch_kernel = resolve_kernel(b->kernel, b->prec == LBM_FP64, any_full, any_hazi, all_tmaps, b->cols);
  const long long slots = step_wave_slots(b->prec == LBM_FP64, b->thermal, b->cols, launch_kernel);
  // every member's tall bands first, then every member's short bands (a member's tile
  // indices, which fix its partial-sum order, are those of the member alone)
  std::vector<Tile> shorts;
  std::vector<FlowInst> flows;
  bool flow_ok = true;
  long long cells = 0;
  for (Member& m : b->slots) {
    if (!m.ctx) continue;
    const int idx = (int)insts.size();
    insts.push_back(lbm_internal_inst(m.ctx));
    m.gen = lbm_internal_params_gen(m.ctx);
    const BandPlan plan = member_plan(b, m.nx, m.ny, slots, total > 0.0 ? (double)m.nx * m.ny / total : 1.0);
    const int strips = (m.nx + w - 1) / w;
    const int y_short = plan.tall_count * plan.tall_rows;
    const int n = strips * (plan.tall_count + (m.ny - y_short + plan.short_rows - 1) / plan.short_rows);
    int local = 0;
    FlowInst f{};
    f.strips = strips;
    f.nbands = n / strips;
    f.tile_w = w;
    f.tall_rows = plan.tall_rows;
    f.tall_count = plan.tall_count;
    f.short_rows = plan.short_rows;
    f.perx = insts[idx].geometry != GEOM_CHANNEL;
    f.pery = insts[idx].geometry == GEOM_PERIODIC;
    f.cell_base = cells;
    cells += n;
    flow_ok = flow_ok && insts[idx].geometry != GEOM_POOL && m.nx >= 3;
    auto band = [&](int y0, int y1, std::vector<Tile>& out) {
      for (int sx = 0; sx < strips; ++sx) {
        Tile t{};
        t.inst = idx;
        t.x0 = sx * w;
        t.y0 = y0;
        t.y1 = y1;
        t.local = local++;
        t.ntiles = n;
        t.interior = tile_is_interior(insts[idx].geometry, m.nx, b->cols, t.x0);
        t.open_end = insts[idx].geometry == GEOM_CHANNEL && (t.x0 == 0 || t.x0 + w >= m.nx);
        f.n_open += t.open_end;
        out.push_back(t);
      }
    };
    for (int bd = 0; bd < plan.tall_count; ++bd) band(bd * plan.tall_rows, (bd + 1) * plan.tall_rows, tiles);
    for (int y = y_short; y < m.ny; y += plan.short_rows) band(y, std::min(m.ny, y + plan.short_rows), shorts);
    flows.push_back(f);
  }
  // the general-loop tiles first (tall bands, then short), then the interior ones
  tiles.insert(tiles.end(), shorts.begin(), shorts.end());
  std::stable_partition(tiles.begin(), tiles.end(), general_tile);
  if (insts.size() > b->cap_insts) {
    if (b->d_insts) cudaFree(b->d_insts);
    if (b->d_flow) cudaFree(b->d_flow);
    if (b->d_step0) cudaFree(b->d_step0);
    b->d_insts = nullptr;
    b->d_flow = nullptr;
    b->d_step0 = nullptr;
    b->cap_insts = std::max<size_t>(insts.size(), 2 * b->cap_insts);
    if (cudaMalloc(&b->d_insts, b->cap_insts * sizeof(Inst)) != cudaSuccess ||
        cudaMalloc(&b->d_flow, b->cap_insts * sizeof(FlowInst)) != cudaSuccess ||
        cudaMalloc(&b->d_step0, b->cap_insts * sizeof(long long)) != cudaSuccess) {
      b->cap_insts = 0;
      return bfail(b, LBM_ENOMEM, "batch descriptor table");
    }
  }
  if (tiles.size() > b->cap_tiles) {
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->d_cells) cudaFree(b->d_cells);
    b->d_tiles = nullptr;
    b->d_cells = nullptr;
    b->cap_tiles = std::max<size_t>(tiles.size(), 2 * b->cap_tiles);
    if (cudaMalloc(&b->d_tiles, b->cap_tiles * sizeof(Tile)) != cudaSuccess ||
        cudaMalloc(&b->d_cells, b->cap_tiles * sizeof(unsigned long long)) != cudaSuccess) {
      b->cap_tiles = 0;
      return bfail(b, LBM_ENOMEM, "batch tile table");
    }
  }
  if (!insts.empty()) {
    LBM_BCUDA(b, cudaMemcpyAsync(b->d_insts, insts.data(), insts.size() * sizeof(Inst), cudaMemcpyHostToDevice,
                                 b->stream));
    LBM_BCUDA(b, cudaMemcpyAsync(b->d_tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice,
                                 b->stream));
    LBM_BCUDA(b, cudaMemcpyAsync(b->d_flow, flows.data(), flows.size() * sizeof(FlowInst), cudaMemcpyHostToDevice,
                                 b->stream));
  }
  b->flow_ok = flow_ok && !insts.empty();
  LBM_BCUDA(b, cudaStreamSynchronize(b->stream));
  b->ntiles = (int)tiles.size();
  b->launch_kernel = launch_kernel;
  b->any_full = any_full;
  drop_graph(b);
  b->dirty = false;
  return LBM_OK;
}

lbm_status launch_steps(lbm_batch* b, int64_t n) {
  for (int64_t k = 0; k < n; ++k) {
    LBM_BCUDA(b, launch_lbm(b->prec == LBM_FP64, b->thermal, b->cols, MODE_STEP, b->launch_kernel, b->any_full,
                            b->d_insts, b->d_tiles, b->ntiles, b->stream, nullptr, b->max_polls));
    ++b->launches;
  }
  return LBM_OK;
}

// CTAs one persistent launch of the batch may hold.
long long batch_slots(const lbm_batch* b) {
  return persistent_slots(b->prec == LBM_FP64, b->thermal, b->cols, b->launch_kernel, b->any_full, false);
}

// Whether the batch's persistent launch overlaps consecutive steps (FlowPlan): every member
// may, and the tiling has more tiles than CTA slots.
bool batch_overlapped(const lbm_batch* b) { return b->flow_ok && b->ntiles > batch_slots(b); }

// Whether a multi-step call takes the persistent launch: on request, or (LBM_LOOP_AUTO) where
// it overlaps the steps of at least two and a half waves of tiles.  With fewer tiles the
// graph-replayed launches measured faster (served mixes of a few lattices: p50 time to result
// 1.86 s against 1.97 s with a barrier between steps).
bool batch_persistent(lbm_batch* b) {
  if (b->launch_kernel != LBM_KERNEL_SCALAR && b->launch_kernel != LBM_KERNEL_INTERIOR) return false;
  if (b->loop == LBM_LOOP_PERSISTENT) return true;
  if (b->loop == LBM_LOOP_LAUNCHES) return false;
  return b->flow_ok && 2 * (long long)b->ntiles >= 5 * batch_slots(b);
}

lbm_status launch_persistent_steps(lbm_batch* b, int64_t nsteps) {
  NvtxRange nvtx("pplbm batch persistent launch");
  if (!b->d_bar && cudaMalloc(&b->d_bar, sizeof(GridBar)) != cudaSuccess) {
    b->d_bar = nullptr;
    return bfail(b, LBM_ENOMEM, "grid barrier of the persistent launch");
  }
  for (int64_t done = 0; done < nsteps;) {
    const int n = (int)std::min<int64_t>(nsteps - done, 1 << 30);
    LBM_BCUDA(b, cudaMemsetAsync(b->d_bar, 0, sizeof(GridBar), b->stream));
    FlowPlan flow{};
    if (batch_overlapped(b)) {
      flow.enabled = 1;
      flow.ninst = 0;
      for (const Member& m : b->slots) flow.ninst += m.ctx != nullptr;
      flow.inst = b->d_flow;
      flow.step0 = b->d_step0;
      flow.cell_done = b->d_cells;
      LBM_BCUDA(b, cudaMemsetAsync(b->d_cells, 0, (size_t)b->ntiles * sizeof(unsigned long long), b->stream));
    }
    LBM_BCUDA(b, launch_persistent(b->prec == LBM_FP64, b->thermal, b->cols, b->launch_kernel, b->any_full, b->d_insts,
                                   b->d_tiles, b->ntiles, n, b->d_bar, b->max_polls, b->stream, nullptr, flow));
    ++b->launches;
    done += n;
  }
  return LBM_OK;
}

lbm_status capture_graph(lbm_batch* b) {
  cudaGraph_t g = nullptr;
  LBM_BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
  lbm_status s = LBM_OK;
  for (int k = 0; k < kGraphChunk && s == LBM_OK; ++k) {
    if (launch_lbm(b->prec == LBM_FP64, b->thermal, b->cols, MODE_STEP, b->launch_kernel, b->any_full, b->d_insts,
                   b->d_tiles, b->ntiles, b->stream, nullptr, b->max_polls) != cudaSuccess)
      s = bfail(b, LBM_ECUDA, "launch during graph capture");
  }
  const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  if (s != LBM_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return bfail(b, LBM_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  const cudaError_t ei = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    b->graph = nullptr;
    return bfail(b, LBM_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ei));
  }
  return LBM_OK;
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(lbm_batch** out, lbm_precision prec, int32_t thermal, int32_t device, void* cuda_stream) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if ((prec != LBM_FP32 && prec != LBM_FP64) || (thermal != 0 && thermal != 1)) return LBM_EINVAL;
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_ENOMEM;
  b->prec = prec;
  b->thermal = thermal;
  b->device = device;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(device) != cudaSuccess) {
    delete b;
    return LBM_ECUDA;
  }
  if (cuda_stream) {
    b->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      if (prev >= 0) cudaSetDevice(prev);
      return LBM_ECUDA;
    }
    b->own_stream = true;
  }
  if (prev >= 0) cudaSetDevice(prev);
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_add(lbm_batch* b, int32_t nx, int32_t ny, const lbm_params* p, int32_t* slot) {
  if (!b || !slot) return LBM_EINVAL;
  if (!p || p->thermal != b->thermal) return bfail(b, LBM_EINVAL, "member must match the batch's thermal flag");
  lbm_ctx* c = nullptr;
  lbm_status s = lbm_create(&c, nx, ny, b->prec, b->device, b->stream);
  if (s != LBM_OK) return bfail(b, s, "member creation failed");
  s = lbm_set_params(c, p);
  if (s != LBM_OK) {
    b->err = lbm_last_error(c);
    lbm_destroy(c);
    return s;
  }
  int idx = -1;
  for (size_t i = 0; i < b->slots.size(); ++i)
    if (!b->slots[i].ctx) {
      idx = (int)i;
      break;
    }
  if (idx < 0) {
    idx = (int)b->slots.size();
    b->slots.push_back(Member{});
  }
  b->slots[idx].ctx = c;
  b->slots[idx].nx = nx;
  b->slots[idx].ny = ny;
  b->dirty = true;
  *slot = idx;
  return LBM_OK;
}

lbm_status lbm_batch_remove(lbm_batch* b, int32_t slot) {
  if (!b || slot < 0 || slot >= (int32_t)b->slots.size() || !b->slots[slot].ctx) return bfail(b, LBM_EINVAL, "no such slot");
  cudaStreamSynchronize(b->stream);
  lbm_destroy(b->slots[slot].ctx);
  b->slots[slot] = Member{};
  b->dirty = true;
  return LBM_OK;
}

lbm_ctx* lbm_batch_member(lbm_batch* b, int32_t slot) {
  if (!b || slot < 0 || slot >= (int32_t)b->slots.size()) return nullptr;
  return b->slots[slot].ctx;
}

int32_t lbm_batch_size(const lbm_batch* b) {
  if (!b) return 0;
  int32_t n = 0;
  for (const Member& m : b->slots) n += m.ctx != nullptr;
  return n;
}

lbm_status lbm_batch_set_tiling(lbm_batch* b, int32_t cols, int32_t rows) {
  if (!b) return LBM_EINVAL;
  if (cols == 0) cols = 128;
  if (!cols_supported(cols)) return bfail(b, LBM_EINVAL, "cols must be 64, 128 or 256");
  if (rows < 0 || (rows > 0 && rows < 4)) return bfail(b, LBM_EINVAL, "rows must be 0 (per-member default) or >= 4");
  b->cols = cols;
  b->rows = rows;
  b->dirty = true;
  return LBM_OK;
}

lbm_status lbm_batch_set_kernel(lbm_batch* b, int32_t kernel) {
  if (!b) return LBM_EINVAL;
  if (kernel < LBM_KERNEL_AUTO || kernel > LBM_KERNEL_INTERIOR)
    return bfail(b, LBM_EINVAL, "kernel must be LBM_KERNEL_AUTO, _SCALAR, _PAIRED, _TMA or _INTERIOR");
  b->kernel = kernel;
  b->dirty = true;  // default band heights depend on the kernel's occupancy; the graph names the kernel
  return LBM_OK;
}

lbm_status lbm_batch_get_tiling(const lbm_batch* b, int32_t* cols, int32_t* rows) {
  if (!b || !cols || !rows) return LBM_EINVAL;
  *cols = b->cols;
  *rows = b->rows;
  return LBM_OK;
}

lbm_status lbm_batch_step_async(lbm_batch* b, int64_t nsteps) {
  NvtxRange nvtx("pplbm batch chunk");
  if (!b || nsteps < 0) return LBM_EINVAL;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  lbm_status s = LBM_OK;
  for (const Member& m : b->slots)  // a member's parameters or state were replaced directly
    if (m.ctx && m.gen != lbm_internal_params_gen(m.ctx)) b->dirty = true;
  if (b->dirty) s = rebuild(b);
  if (s == LBM_OK && b->ntiles > 0 && nsteps >= 2 && batch_persistent(b)) {
    s = launch_persistent_steps(b, nsteps);
  } else if (s == LBM_OK && b->ntiles > 0) {
    int64_t left = nsteps;
    if (left >= kGraphChunk && !b->graph) s = capture_graph(b);
    while (s == LBM_OK && left >= kGraphChunk) {
      const cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
      if (e != cudaSuccess) s = bfail(b, LBM_ECUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
      b->launches += kGraphChunk;
      left -= kGraphChunk;
    }
    if (s == LBM_OK) s = launch_steps(b, left);
  }
  if (prev >= 0) cudaSetDevice(prev);
  return s;
}

lbm_status lbm_batch_set_step_loop(lbm_batch* b, int32_t loop) {
  if (!b) return LBM_EINVAL;
  if (loop < LBM_LOOP_AUTO || loop > LBM_LOOP_PERSISTENT)
    return bfail(b, LBM_EINVAL, "loop must be LBM_LOOP_AUTO, _LAUNCHES or _PERSISTENT");
  b->loop = loop;
  return LBM_OK;
}

int32_t lbm_batch_step_loop(lbm_batch* b) {
  if (!b) return -1;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  int32_t out = -1;
  if (!b->dirty || rebuild(b) == LBM_OK)
    out = !batch_persistent(b) ? LBM_LOOP_LAUNCHES : (batch_overlapped(b) ? LBM_LOOP_OVERLAPPED : LBM_LOOP_PERSISTENT);
  if (prev >= 0) cudaSetDevice(prev);
  return out;
}

lbm_status lbm_batch_set_wait_limit(lbm_batch* b, int64_t max_polls) {
  if (!b) return LBM_EINVAL;
  if (max_polls < 0 || max_polls > 0xffffffffll) return bfail(b, LBM_EINVAL, "max_polls out of range");
  b->max_polls = (unsigned)max_polls;
  return LBM_OK;
}

lbm_status lbm_batch_sync(lbm_batch* b, int32_t* unstable_slot) {
  if (!b) return LBM_EINVAL;
  if (unstable_slot) *unstable_slot = -1;
  lbm_status worst = LBM_OK;
  for (size_t i = 0; i < b->slots.size(); ++i) {
    if (!b->slots[i].ctx) continue;
    const lbm_status s = lbm_sync(b->slots[i].ctx);
    if (s != LBM_OK && worst == LBM_OK) {
      worst = s;
      b->err = lbm_last_error(b->slots[i].ctx);
      if (unstable_slot) *unstable_slot = (int32_t)i;
    }
  }
  return worst;
}

lbm_status lbm_batch_step(lbm_batch* b, int64_t nsteps) {
  const lbm_status s = lbm_batch_step_async(b, nsteps);
  if (s != LBM_OK) return s;
  return lbm_batch_sync(b, nullptr);
}

lbm_status lbm_batch_read_fields(lbm_batch* b, int32_t slot, double* rho, double* ux, double* uy, double* T,
                                 size_t n) {
  lbm_ctx* c = lbm_batch_member(b, slot);
  if (!c) return bfail(b, LBM_EINVAL, "no such slot");
  return lbm_read_fields(c, rho, ux, uy, T, n);
}

lbm_status lbm_batch_autotune(lbm_batch* b, int32_t trial_steps, int32_t* cols_out, int32_t* rows_out) {
  if (!b || trial_steps < 1) return LBM_EINVAL;
  static const int kCols[] = {64, 128, 256};
  static const int kRows[] = {0, 16, 24, 32, 48, 64};
  cudaEvent_t e0, e1;
  LBM_BCUDA(b, cudaEventCreate(&e0));
  LBM_BCUDA(b, cudaEventCreate(&e1));
  float best = -1.0f;
  int best_c = b->cols, best_r = b->rows;
  lbm_status s = LBM_OK;
  for (int c : kCols) {
    for (int r : kRows) {
      if ((s = lbm_batch_set_tiling(b, c, r)) != LBM_OK) break;
      if ((s = lbm_batch_step_async(b, 2)) != LBM_OK) break;  // warm-up and table upload
      cudaEventRecord(e0, b->stream);
      if ((s = lbm_batch_step_async(b, trial_steps)) != LBM_OK) break;
      cudaEventRecord(e1, b->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        s = bfail(b, LBM_ECUDA, "autotune timing");
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (best < 0.0f || ms < best) {
        best = ms;
        best_c = c;
        best_r = r;
      }
    }
    if (s != LBM_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != LBM_OK) return s;
  lbm_batch_set_tiling(b, best_c, best_r);
  if (cols_out) *cols_out = best_c;
  if (rows_out) *rows_out = best_r;
  return lbm_batch_sync(b, nullptr);
}

int64_t lbm_batch_launch_count(const lbm_batch* b) { return b ? b->launches : -1; }

void* lbm_batch_get_stream(const lbm_batch* b) { return b ? static_cast<void*>(b->stream) : nullptr; }

const char* lbm_batch_last_error(const lbm_batch* b) { return b ? b->err.c_str() : "NULL batch"; }

lbm_status lbm_batch_destroy(lbm_batch* b) {
  if (!b) return LBM_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  for (Member& m : b->slots)
    if (m.ctx) lbm_destroy(m.ctx);
  if (b->d_insts) cudaFree(b->d_insts);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->d_bar) cudaFree(b->d_bar);
  if (b->d_flow) cudaFree(b->d_flow);
  if (b->d_step0) cudaFree(b->d_step0);
  if (b->d_cells) cudaFree(b->d_cells);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  if (prev >= 0) cudaSetDevice(prev);
  delete b;
  return LBM_OK;
}

}  // extern "C"
