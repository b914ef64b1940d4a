// Host side of the pplbm C ABI: contexts, parameter validation, device memory
// layout, launches and readback.  Every exported function returns a status and
// never throws.
#include <cuda.h>  // CUtensorMap and its encoder's types (the encoder is fetched at run time)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lbm_internal.h"
#include "pplbm.h"

namespace pplbm {
cudaError_t launch_lbm_f32(int, int, int, int, bool, const Inst*, const Tile*, int, cudaStream_t, const Inst*,
                          unsigned);
cudaError_t launch_lbm_f64(int, int, int, int, bool, const Inst*, const Tile*, int, cudaStream_t, const Inst*);
cudaError_t launch_init_from_fields_f32(const Inst*, int, int, const double*, int, cudaStream_t);
cudaError_t launch_init_from_fields_f64(const Inst*, int, int, const double*, int, cudaStream_t);
cudaError_t launch_init_builtin_f32(const Inst*, int, int, InitSpec, cudaStream_t);
cudaError_t launch_init_builtin_f64(const Inst*, int, int, InitSpec, cudaStream_t);

cudaError_t launch_persistent_f32(int, int, int, bool, const Inst*, const Tile*, int, int, GridBar*, unsigned,
                                  cudaStream_t, const Inst*, const FlowPlan&);
cudaError_t launch_persistent_f64(int, int, int, bool, const Inst*, const Tile*, int, int, GridBar*, unsigned,
                                  cudaStream_t, const Inst*, const FlowPlan&);
int persistent_resident_f32(int, int, int, bool, bool);
int persistent_resident_f64(int, int, int, bool, bool);

cudaError_t launch_persistent(int fp64, int thermal, int cols, int kernel, bool full, const Inst* d_inst,
                              const Tile* d_tiles, int ntiles, int nsteps, GridBar* bar, unsigned max_polls,
                              cudaStream_t s, const Inst* h_inst, const FlowPlan& flow) {
  return fp64 ? launch_persistent_f64(thermal, cols, kernel, full, d_inst, d_tiles, ntiles, nsteps, bar, max_polls, s,
                                      h_inst, flow)
              : launch_persistent_f32(thermal, cols, kernel, full, d_inst, d_tiles, ntiles, nsteps, bar, max_polls, s,
                                      h_inst, flow);
}

long long persistent_slots(int fp64, int thermal, int cols, int kernel, bool full, bool single) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = fp64 ? persistent_resident_f64(thermal, cols, kernel, full, single)
                          : persistent_resident_f32(thermal, cols, kernel, full, single);
  return (long long)sms * per_sm;
}

cudaError_t launch_lbm(int fp64, int thermal, int cols, int mode, int kernel, bool full, const Inst* d_inst,
                       const Tile* d_tiles, int ntiles, cudaStream_t s, const Inst* h_inst, unsigned max_polls) {
  return fp64 ? launch_lbm_f64(thermal, cols, mode, kernel, full, d_inst, d_tiles, ntiles, s, h_inst)
              : launch_lbm_f32(thermal, cols, mode, kernel, full, d_inst, d_tiles, ntiles, s, h_inst, max_polls);
}
cudaError_t launch_init_from_fields(int fp64, const Inst* d_inst, int nx, int ny, const double* d_fields,
                                    int has_T, cudaStream_t s) {
  return fp64 ? launch_init_from_fields_f64(d_inst, nx, ny, d_fields, has_T, s)
              : launch_init_from_fields_f32(d_inst, nx, ny, d_fields, has_T, s);
}
cudaError_t launch_init_builtin(int fp64, const Inst* d_inst, int nx, int ny, InitSpec spec, cudaStream_t s) {
  return fp64 ? launch_init_builtin_f64(d_inst, nx, ny, spec, s) : launch_init_builtin_f32(d_inst, nx, ny, spec, s);
}
bool cols_supported(int cols) { return cols == 64 || cols == 128 || cols == 256; }

const char* check_params(int nx, int ny, const lbm_params* p) {
  if (!p) return "params is NULL";
  if (p->size != sizeof(lbm_params)) return "params.size != sizeof(lbm_params)";
  if (p->geometry < 0 || p->geometry > 3) return "geometry must be 0, 1, 2 or 3";
  if (p->source_model != LBM_SOURCE_GONG_CHENG && p->source_model != LBM_SOURCE_HAZI_MARKUS)
    return "source_model must be LBM_SOURCE_GONG_CHENG or LBM_SOURCE_HAZI_MARKUS";
  if (p->bubble_stats != 0 && p->bubble_stats != 1) return "bubble_stats must be 0 or 1";
  if (p->geometry == LBM_GEOM_POOL && ny < 3) return "pool geometry needs ny >= 3";
  if (p->geometry == LBM_GEOM_POOL && !(p->rho_out > 0)) return "pool geometry needs rho_out > 0";
  if (p->geometry == LBM_GEOM_CHANNEL && (nx < 3 || ny < 2)) return "channel needs nx >= 3 and ny >= 2";
  if (p->geometry == LBM_GEOM_WALLS && ny < 2) return "walls geometry needs ny >= 2";
  if (p->thermal != 0 && p->thermal != 1) return "thermal must be 0 or 1";
  if (p->multiphase != 0 && p->multiphase != 1) return "multiphase must be 0 or 1";
  if (!(p->tau_f > 0.5) || !(p->tau_g > 0.5)) return "tau_f and tau_g must exceed 1/2";
  if (!(p->a > 0) || !(p->b > 0) || !(p->R > 0)) return "a, b, R must be positive";
  if (!(p->T0_R > 0) || !(p->Tin_R > 0) || !(p->Tin_R + p->dTheat_R > 0)) return "temperatures must be positive";
  if (p->multiphase && (!(p->c0 > 0) || p->G == 0.0 || !std::isfinite(p->G))) return "c0 > 0 and G != 0 required";
  if (p->thermal && !(p->c_v > 0)) return "c_v must be positive";
  if (p->geometry == LBM_GEOM_CHANNEL && (!(p->rho_out > 0) || !(std::fabs(p->u_in) < 0.5)))
    return "rho_out > 0 and |u_in| < 0.5 required";
  if (p->heater_len < 0) return "heater_len must be >= 0";
  if (p->init_kind != LBM_INIT_UNIFORM && p->init_kind != LBM_INIT_DISK) return "init_kind must be 0 or 1";
  if (!(p->init_rho_out > 0) || (p->init_kind == LBM_INIT_DISK && (!(p->init_rho_in > 0) || !(p->init_width > 0))))
    return "initial densities and width must be positive";
  if (!std::isfinite(p->u_in) || !std::isfinite(p->g_a) || !std::isfinite(p->G_wet) || !std::isfinite(p->beta))
    return "non-finite parameter";
  return nullptr;
}

namespace {
// Peng-Robinson pressure (Eq. 12) in double on the host, for psi(rho_w, T0).
double host_pressure(const lbm_params& p, double rho, double T) {
  const double Tc = 0.0778 * p.a / (0.45724 * p.b * p.R);
  const double kappa = 0.37464 + 1.54226 * p.omega - 0.26992 * p.omega * p.omega;
  const double s = 1.0 + kappa * (1.0 - std::sqrt(T / Tc));
  return rho * p.R * T / (1.0 - p.b * rho) - p.a * s * s * rho * rho / (1.0 + 2.0 * p.b * rho - p.b * p.b * rho * rho);
}
}  // namespace

const char* fill_inst(Inst& I, const lbm_params* p, int nx, int ny, int pitch, long long plane, int fp64) {
  I = Inst{};
  I.nx = nx;
  I.ny = ny;
  I.pitch = pitch;
  I.geometry = p->geometry;
  I.plane = plane;
  for (int j = 0; j < NPART; ++j) {
    // nodes feeding total j: the heater row (2), the inlet and outlet columns (3, 4), else all
    const long long m = j == 2 ? nx : (j == 3 || j == 4) ? ny : (long long)nx * ny;
    int e = 0;  // ceil(log2(m))
    while ((1ll << e) < m) ++e;
    I.fix_scale[j] = std::ldexp(1.0, FIX_BITS - e);
    I.fix_unscale[j] = std::ldexp(1.0, e - FIX_BITS);
  }
  I.multiphase = p->multiphase;
  I.omega_f = 1.0 / p->tau_f;
  I.omega_g = 1.0 / p->tau_g;
  const double Tc = 0.0778 * p->a / (0.45724 * p->b * p->R);
  I.a = p->a;
  I.b = p->b;
  I.R = p->R;
  I.kappa = 0.37464 + 1.54226 * p->omega - 0.26992 * p->omega * p->omega;
  I.sqrtTc = std::sqrt(Tc);
  I.inv_sqrtTc = 1.0 / I.sqrtTc;
  I.T0 = p->T0_R * Tc;
  I.T_in = p->Tin_R * Tc;
  I.T_heat = (p->Tin_R + p->dTheat_R) * Tc;
  {
    const double sa = 1.0 + I.kappa * (1.0 - std::sqrt(I.T0 / Tc));
    I.alpha0 = sa * sa;
  }
  if (p->multiphase) {
    I.psi_scale = 2.0 / (p->c0 * p->G);
    const double rad = (host_pressure(*p, p->rho_w, I.T0) - p->rho_w / 3.0) * I.psi_scale;
    if (!(rad >= 0.0)) return "psi(rho_w, T0) undefined: negative radicand (Eq. 11)";
    I.Gwet_psiw = p->G_wet * std::sqrt(rad);
    if (!(p->b * std::max(p->rho_w, p->init_rho_out) < 1.0)) return "density beyond 1/b";
  }
  I.beta = p->beta;
  I.G2 = 2.0 * p->G;
  I.Ghalf = 0.5 * p->G;
  I.g_a = p->g_a;
  I.inv_cv = p->thermal ? 1.0 / p->c_v : 0.0;
  I.u_in = p->u_in;
  I.rho_out = p->rho_out;
  if (!fp64) {
    I.rho_ref = p->geometry == LBM_GEOM_CHANNEL ? p->rho_out : p->init_rho_out;
    I.T_ref = I.T0;
  } else {
    I.rho_ref = 0.0;
    I.T_ref = 0.0;
  }
  if (!fp64 && p->multiphase) {
    const double rr = I.rho_ref, Tr = I.T_ref;
    const double u1r = 1.0 - p->b * rr, Dr = 1.0 + 2.0 * p->b * rr - p->b * p->b * rr * rr;
    if (!(u1r > 0.0) || !(Dr > 0.0)) return "reference density beyond 1/b";
    I.sa_r = 1.0 + I.kappa * (1.0 - std::sqrt(Tr / Tc));
    I.p_ref = rr * p->R * Tr / u1r - p->a * I.sa_r * I.sa_r * rr * rr / Dr;
    I.rad_ref = (I.p_ref - rr / 3.0) * I.psi_scale;
    if (!(I.rad_ref >= 0.0)) return "psi undefined at the reference state (Eq. 11)";
    I.psi_ref = std::sqrt(I.rad_ref);
    I.inv_u1r = 1.0 / u1r;
    I.inv_Dr = 1.0 / Dr;
    I.sqrtT_r = std::sqrt(Tr);
    I.rr2_Dr = rr * rr / Dr;
  }
  for (int i = 0; i < 9; ++i) {
    static const int cx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, cy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
    I.poff[i] = (int)(i * plane);
    I.loff[i] = (int)(i * plane - cy[i] * (long long)pitch - cx[i]);
  }
  I.mix = 0.5 * (1.0 - I.beta);
  I.drho_out = I.rho_out - I.rho_ref;
  I.dT_in = I.T_in - I.T_ref;
  I.dT_heat = I.T_heat - I.T_ref;
  I.drho_vapor = p->rho_vapor - I.rho_ref;
  {
    const double G3 = 1.5 * I.G2, pr = I.psi_ref;
    I.wall0 = -G3 * (I.beta + I.mix) * pr * pr + I.Gwet_psiw * pr / 6.0;
    I.wall1 = -G3 * I.beta * pr + I.Gwet_psiw / 6.0;
  }
  I.R_u1r = I.R * I.inv_u1r;
  I.a_Dr = I.a * I.inv_Dr;
  I.twob_rr = 2.0 * I.b * I.rho_ref;
  I.nk_sTc = -I.kappa * I.inv_sqrtTc;
  I.a_rr2_Dr = I.a * I.rr2_Dr;
  I.heater_x0 = p->heater_x0 < 0 ? nx / 5 : p->heater_x0;
  I.heater_len = p->heater_len;
  I.heat_on_step = p->heat_on_step;
  I.rho_vapor = p->rho_vapor;
  I.source_model = p->source_model;
  I.bubble_stats = p->bubble_stats;
  return nullptr;
}

int default_band_rows(int nx, int ny, int cols, long long slots) {
  const int w = cols - 8;
  const long long strips = (nx + w - 1) / w;
  if (slots < 1) slots = 1;
  if (ny <= 4) return ny;
  int best_rows = ny;
  double best_cost = -1.0;
  // candidate band counts: every distinct balanced band height from ny down to 4 rows
  for (int bands = 1; bands <= ny; ++bands) {
    const int rows = (ny + bands - 1) / bands;
    if (rows < 4) break;
    if (bands > 1 && rows == (ny + bands - 2) / (bands - 1)) continue;  // same height as bands - 1
    const long long tiles = strips * ((ny + rows - 1) / rows);
    // row-iterations per CTA slot: the work spread over all slots plus, with the block
    // scheduler refilling slots as tiles finish, about half a tile of tail
    const double cost = (double)tiles * (rows + 5) / (double)slots + 0.5 * (rows + 5);
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best_rows = rows;
    }
  }
  return best_rows;
}

BandPlan default_band_plan(int nx, int ny, int cols, long long slots) {
  const int rows = default_band_rows(nx, ny, cols, slots);
  BandPlan best{0, 0, rows};
  const int w = cols - 8;
  const long long strips = (nx + w - 1) / w;
  if (slots < 1) slots = 1;
  // the cost model of default_band_rows: row-iterations per CTA slot = the work (rows + 4 halo
  // rows + about one row of fixed cost per tile) spread over the slots, plus half of a tile of
  // the class dispatched last
  const long long ubands = (ny + rows - 1) / rows;
  double best_cost = (double)(strips * ubands) * (rows + 5) / (double)slots + 0.5 * (rows + 5);
  const long long ks = (slots + strips - 1) / strips;  // short bands per strip: about one wave of short tiles
  for (int h = 4; (ks + 2) * h <= ny; ++h) {
    const int tall = (int)((ny - ks * h) / (2 * h));
    double work = (double)strips * tall * (2 * h + 5);
    for (int y = tall * 2 * h; y < ny; y += h) work += (double)strips * (std::min(h, ny - y) + 5);
    const double cost = work / (double)slots + 0.5 * (h + 5);
    if (cost < best_cost) {
      best_cost = cost;
      best = BandPlan{2 * h, tall, h};
    }
  }
  return best;
}

long long step_wave_slots(int fp64, int thermal, int cols, int kernel) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = fp64 ? resident_ctas_f64(thermal, cols, kernel) : resident_ctas_f32(thermal, cols, kernel);
  return (long long)sms * (per_sm > 0 ? per_sm : 1);
}
}  // namespace pplbm

using namespace pplbm;

namespace {

constexpr int kAuxCols = 128;       // tile width of the field/population readback passes
constexpr int kAuxRows = 32;
constexpr int kMinRows = 4;          // smallest band a step tiling may use
constexpr size_t kAlign = 256;
constexpr int kMaxDim = 1 << 20;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  int pitch;
  long long plane;
  size_t pop_bytes;  // one 9-plane buffer
  int max_tiles;
  size_t off_f[2], off_g[2], off_rho_prev, off_tmaps, off_inst, off_state, off_sums, off_bar, off_cells, off_step0, off_ring,
      off_tiles_step, off_tiles_aux, total;
};

Layout make_layout(int nx, int ny, lbm_precision prec) {
  Layout L{};
  const size_t elt = prec == LBM_FP64 ? 8 : 4;
  L.pitch = (nx + 31) / 32 * 32;
  L.plane = (long long)L.pitch * ny;
  L.pop_bytes = align_up(9 * (size_t)L.plane * elt);
  const long long strips = (nx + 55) / 56;  // narrowest tiling: 64 threads, 56 output columns
  const long long bands = (ny + kMinRows - 1) / kMinRows;
  L.max_tiles = (int)std::min<long long>(strips * bands, 1ll << 30);
  size_t off = 0;
  for (int b = 0; b < 2; ++b) { L.off_f[b] = off; off += L.pop_bytes; }
  for (int b = 0; b < 2; ++b) { L.off_g[b] = off; off += L.pop_bytes; }
  L.off_rho_prev = off; off += align_up((size_t)L.plane * elt);
  L.off_tmaps = off; off += align_up(4 * sizeof(CUtensorMap));
  L.off_inst = off; off += align_up(sizeof(Inst));
  L.off_state = off; off += align_up(sizeof(InstState));
  L.off_sums = off; off += align_up(2 * NPART * sizeof(unsigned long long));  // two steps' totals
  L.off_bar = off; off += align_up(sizeof(GridBar));
  L.off_cells = off; off += align_up((size_t)L.max_tiles * sizeof(unsigned long long));  // overlapped loop
  L.off_step0 = off; off += align_up(sizeof(long long));
  L.off_ring = off; off += align_up((size_t)RING * NDIAG * sizeof(double));
  L.off_tiles_step = off; off += align_up((size_t)L.max_tiles * sizeof(Tile));
  L.off_tiles_aux = off; off += align_up((size_t)L.max_tiles * sizeof(Tile));
  L.total = off;
  return L;
}

// Output columns of one tile: a CTA of `cols` threads writes cols - 8 columns.
int tile_cols(int cols) { return cols - 8; }

// Tiles of a band plan in dispatch order: the tall bands of every strip (band by band),
// then the short bands.
void build_tiles(int nx, int ny, int cols, const BandPlan& plan, std::vector<Tile>& out, int geometry) {
  out.clear();
  const int w = tile_cols(cols);
  const int strips = (nx + w - 1) / w;
  auto band = [&](int y0, int y1) {
    for (int sidx = 0; sidx < strips; ++sidx) {
      Tile t{};
      t.inst = 0;
      t.x0 = sidx * w;
      t.y0 = y0;
      t.y1 = y1;
      t.interior = tile_is_interior(geometry, nx, cols, t.x0);
      t.open_end = geometry == GEOM_CHANNEL && (t.x0 == 0 || t.x0 + w >= nx);
      out.push_back(t);
    }
  };
  for (int b = 0; b < plan.tall_count; ++b) band(b * plan.tall_rows, (b + 1) * plan.tall_rows);
  for (int y = plan.tall_count * plan.tall_rows; y < ny; y += plan.short_rows)
    band(y, std::min(ny, y + plan.short_rows));
  // The tiles that take the general loop (the strips at the open ends or at a wrap, slower per
  // row than the interior path) first, tall bands before short ones, then the interior tiles
  // of the tall and the short bands: none of the slow tiles is among the last a launch
  // dispatches, and in the overlapped persistent loop the inlet and outlet tiles, whose mass
  // balance every tile of the next step waits for, finish early in their step.
  std::stable_partition(out.begin(), out.end(), general_tile);
  for (size_t k = 0; k < out.size(); ++k) {
    out[k].local = (int)k;
    out[k].ntiles = (int)out.size();
  }
}

// cuTensorMapEncodeTiled, fetched from the driver at run time (the library does not
// link the driver API).  Null when the driver does not provide it.
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// The TMA step kernel's view of one FP32 population buffer: a 3-D tensor (x: nx columns,
// y: ny rows `pitch` apart, z: 9 planes `plane` apart) read in boxes of one 128-column
// row of one plane; boxes reaching outside the tensor read zeros.
bool encode_pop_map(CUtensorMap* m, void* base, int nx, int ny, int pitch, long long plane) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, 9};
  const cuuint64_t strides[2] = {(cuuint64_t)pitch * sizeof(float), (cuuint64_t)plane * sizeof(float)};
  const cuuint32_t box[3] = {(cuuint32_t)TMA_TILE_COLS, 1, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}


}  // namespace

struct lbm_ctx {
  int nx = 0, ny = 0;
  lbm_precision prec = LBM_FP32;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  char* base = nullptr;
  bool own_mem = false;
  Layout L{};
  Inst hinst{};
  Inst* d_inst = nullptr;
  InstState* d_state = nullptr;
  InstState* h_state = nullptr;  // pinned mirror
  int cols = 128, rows = 16;
  BandPlan plan{0, 0, 16};  // the step tiling's bands
  bool rows_default = true;  // band height chosen by default_band_rows (re-chosen on changes)
  int ntiles_step = 0, ntiles_aux = 0;
  int nopen_step = 0;  // step tiles with an open end (inlet or outlet columns)
  Tile* d_tiles_step = nullptr;
  Tile* d_tiles_aux = nullptr;
  lbm_params params{};
  bool have_params = false;
  int thermal = 0;
  long long launches = 0;
  long long step_host = 0;  // step count as last synchronised
  unsigned long long params_gen = 0;  // bumped whenever the descriptor changes
  int kernel = LBM_KERNEL_AUTO;        // requested step kernel form (resolve_kernel picks the one launched)
  int loop = LBM_LOOP_AUTO;            // requested step loop (one launch per step or persistent)
  unsigned max_polls = 0;              // barrier polls before a persistent launch gives up (0: time limit only)
  bool have_tmaps = false;             // FP32: the tensor maps of the population buffers are on the device
  std::string err;
};

namespace {

lbm_status fail(lbm_ctx* c, lbm_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

lbm_status cuda_fail(lbm_ctx* c, cudaError_t e, const char* where) {
  return fail(c, LBM_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define LBM_CUDA(ctx, call)                                   \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);  \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

size_t elt_size(const lbm_ctx* c) { return c->prec == LBM_FP64 ? 8 : 4; }

// A new state (initialisation, injected populations, a loaded checkpoint): the step state,
// and zero totals of the partial sums (a launch that gave up waiting may have left some).
lbm_status upload_state(lbm_ctx* c) {
  LBM_CUDA(c, cudaMemcpyAsync(c->d_state, c->h_state, sizeof(InstState), cudaMemcpyHostToDevice, c->stream));
  LBM_CUDA(c, cudaMemsetAsync(c->base + c->L.off_sums, 0, 2 * NPART * sizeof(unsigned long long), c->stream));
  return LBM_OK;
}

lbm_status fetch_state(lbm_ctx* c) {
  LBM_CUDA(c, cudaMemcpyAsync(c->h_state, c->d_state, sizeof(InstState), cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  c->step_host = c->h_state->step;
  return LBM_OK;
}

lbm_status set_tiling(lbm_ctx* c, int cols, const BandPlan& plan) {
  std::vector<Tile> t;
  // the interior flags depend on the geometry: set_params and load_state rebuild the table
  build_tiles(c->nx, c->ny, cols, plan, t, c->have_params ? c->params.geometry : LBM_GEOM_PERIODIC);
  if ((int)t.size() > c->L.max_tiles) return fail(c, LBM_EINVAL, "tiling needs more tiles than reserved");
  LBM_CUDA(c, cudaMemcpyAsync(c->d_tiles_step, t.data(), t.size() * sizeof(Tile), cudaMemcpyHostToDevice, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  c->cols = cols;
  c->rows = plan.short_rows;
  c->plan = plan;
  c->ntiles_step = (int)t.size();
  c->nopen_step = (int)std::count_if(t.begin(), t.end(), [](const Tile& x) { return x.open_end != 0; });
  return LBM_OK;
}

int step_kernel(const lbm_ctx* c, int cols) {
  return resolve_kernel(c->kernel, c->prec == LBM_FP64, needs_full_step(c->hinst),
                        c->params.source_model == LBM_SOURCE_HAZI_MARKUS, c->have_tmaps, cols);
}

// Re-choose the default tiling for the current kernel, precision and thermal flag.
lbm_status retile_default(lbm_ctx* c, int cols) {
  const long long slots =
      step_wave_slots(c->prec == LBM_FP64, c->have_params ? c->thermal : 1, cols, step_kernel(c, cols));
  const lbm_status s = set_tiling(c, cols, default_band_plan(c->nx, c->ny, cols, slots));
  if (s == LBM_OK) c->rows_default = true;
  return s;
}

// Whether a persistent launch of this context may overlap consecutive steps (FlowPlan): the
// channel, walls and periodic geometries (the mass through the pool's open top is not
// accounted), with distinct inlet and outlet columns.
bool flow_eligible(const lbm_ctx* c) {
  return c->have_params && c->params.geometry != LBM_GEOM_POOL && c->nx >= 3;
}

// Whether a persistent launch of the current tiling overlaps the steps: more tiles than CTAs.
bool overlapped(lbm_ctx* c) {
  if (!flow_eligible(c)) return false;
  const long long slots = persistent_slots(c->prec == LBM_FP64, c->thermal, c->cols, step_kernel(c, c->cols),
                                           needs_full_step(c->hinst), true);
  return c->ntiles_step > slots;
}

// Whether lbm_step_async takes the persistent launch: requested, or (LBM_LOOP_AUTO) when the
// step tiling is one wave of the persistent kernel, where a step's launch gap and kernel
// boundary are a large part of it, or at least two and a half waves that the overlapped form
// can run (the end of each step then overlaps the start of the next; with fewer tiles per CTA
// the next step's first tiles mostly wait, and one launch per step measured faster).  Only
// the one-column kernel (general or interior path) has a persistent form.
bool use_persistent(lbm_ctx* c) {
  if (c->loop == LBM_LOOP_LAUNCHES) return false;
  const int kernel = step_kernel(c, c->cols);
  if (kernel != LBM_KERNEL_SCALAR && kernel != LBM_KERNEL_INTERIOR) return false;
  if (c->loop == LBM_LOOP_PERSISTENT) return true;
  const long long slots = persistent_slots(c->prec == LBM_FP64, c->thermal, c->cols, kernel,
                                           needs_full_step(c->hinst), true);
  return c->ntiles_step <= slots || (flow_eligible(c) && 2 * (long long)c->ntiles_step >= 5 * slots);
}

lbm_status launch(lbm_ctx* c, int mode) {
  const bool step_tiles = mode == MODE_STEP;
  const int kernel = step_tiles ? step_kernel(c, c->cols) : LBM_KERNEL_SCALAR;
  cudaError_t e = launch_lbm(c->prec == LBM_FP64, c->thermal, step_tiles ? c->cols : kAuxCols, mode, kernel,
                             needs_full_step(c->hinst), c->d_inst,
                             step_tiles ? c->d_tiles_step : c->d_tiles_aux,
                             step_tiles ? c->ntiles_step : c->ntiles_aux, c->stream, &c->hinst, c->max_polls);
  if (e != cudaSuccess) return cuda_fail(c, e, "kernel launch");
  ++c->launches;
  return LBM_OK;
}

// Fill the device instance descriptor from validated parameters.
lbm_status apply_params(lbm_ctx* c, const lbm_params* p) {
  if (const char* why = check_params(c->nx, c->ny, p)) return fail(c, LBM_EINVAL, why);
  Inst& I = c->hinst;
  if (const char* why = fill_inst(I, p, c->nx, c->ny, c->L.pitch, c->L.plane, c->prec == LBM_FP64))
    return fail(c, LBM_EINVAL, why);
  for (int b = 0; b < 2; ++b) {
    I.f[b] = c->base + c->L.off_f[b];
    I.g[b] = c->base + c->L.off_g[b];
  }
  I.rho_prev = c->base + c->L.off_rho_prev;
  I.tmaps = c->have_tmaps ? c->base + c->L.off_tmaps : nullptr;
  I.st = c->d_state;
  I.sums = reinterpret_cast<unsigned long long*>(c->base + c->L.off_sums);
  I.ring = reinterpret_cast<double*>(c->base + c->L.off_ring);
  LBM_CUDA(c, cudaMemcpyAsync(c->d_inst, &c->hinst, sizeof(Inst), cudaMemcpyHostToDevice, c->stream));
  c->params = *p;
  c->thermal = p->thermal;
  c->have_params = true;
  ++c->params_gen;
  return LBM_OK;
}

void reset_state_mirror(lbm_ctx* c, long long step, int local, double rho_avg_prev) {
  InstState& S = *c->h_state;
  std::memset(&S, 0, sizeof(S));
  S.step = step;
  S.local_read = local;
  S.rho_avg[(step - 1) & 1] = rho_avg_prev;
  S.rho_avg[step & 1] = rho_avg_prev;
}

lbm_status create_impl(lbm_ctx** out, int32_t nx, int32_t ny, lbm_precision prec, int32_t device, void* stream,
                       void* dev_buf, size_t dev_bytes) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (nx < 1 || ny < 1 || nx > kMaxDim || ny > kMaxDim) return LBM_EINVAL;
  if (prec != LBM_FP32 && prec != LBM_FP64) return LBM_EINVAL;
  if (dev_buf && (reinterpret_cast<uintptr_t>(dev_buf) % kAlign) != 0) return LBM_EINVAL;
  // kernels index one 9-plane population buffer with 32-bit element offsets
  if (9ll * make_layout(nx, ny, prec).plane >= (1ll << 31)) return LBM_EINVAL;
  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return LBM_ENOMEM;
  c->nx = nx;
  c->ny = ny;
  c->prec = prec;
  c->device = device;
  c->L = make_layout(nx, ny, prec);
  DeviceGuard g(device);
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) { delete c; return LBM_ECUDA; }
  if (stream) {
    c->stream = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { delete c; return LBM_ECUDA; }
    c->own_stream = true;
  }
  if (dev_buf) {
    if (dev_bytes < c->L.total) { lbm_destroy(c); return LBM_ENOMEM; }
    c->base = static_cast<char*>(dev_buf);
  } else {
    void* p = nullptr;
    if (cudaMalloc(&p, c->L.total) != cudaSuccess) { cudaGetLastError(); lbm_destroy(c); return LBM_ENOMEM; }
    c->base = static_cast<char*>(p);
    c->own_mem = true;
  }
  if (cudaMallocHost(&c->h_state, sizeof(InstState)) != cudaSuccess) { lbm_destroy(c); return LBM_ENOMEM; }
  std::memset(c->h_state, 0, sizeof(InstState));
  c->d_inst = reinterpret_cast<Inst*>(c->base + c->L.off_inst);
  c->d_state = reinterpret_cast<InstState*>(c->base + c->L.off_state);
  c->d_tiles_step = reinterpret_cast<Tile*>(c->base + c->L.off_tiles_step);
  c->d_tiles_aux = reinterpret_cast<Tile*>(c->base + c->L.off_tiles_aux);
  if (prec == LBM_FP32) {
    // tensor maps of f and g, both buffers, for the TMA step kernel (without them the
    // scalar kernel runs)
    CUtensorMap maps[4];
    bool ok = true;
    for (int b = 0; b < 2; ++b) {
      ok = ok && encode_pop_map(&maps[b], c->base + c->L.off_f[b], nx, ny, c->L.pitch, c->L.plane);
      ok = ok && encode_pop_map(&maps[2 + b], c->base + c->L.off_g[b], nx, ny, c->L.pitch, c->L.plane);
    }
    if (ok) {
      if (cudaMemcpyAsync(c->base + c->L.off_tmaps, maps, sizeof(maps), cudaMemcpyHostToDevice, c->stream) !=
              cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess) {
        lbm_destroy(c);
        return LBM_ECUDA;
      }
      c->have_tmaps = true;
    }
  }
  std::vector<Tile> t;
  build_tiles(nx, ny, kAuxCols, BandPlan{0, 0, std::min(kAuxRows, ny)}, t, LBM_GEOM_PERIODIC);
  c->ntiles_aux = (int)t.size();
  if (cudaMemcpyAsync(c->d_tiles_aux, t.data(), t.size() * sizeof(Tile), cudaMemcpyHostToDevice, c->stream) !=
          cudaSuccess ||
      cudaMemsetAsync(c->base + c->L.off_state, 0, sizeof(InstState), c->stream) != cudaSuccess ||
      cudaMemsetAsync(c->base + c->L.off_sums, 0, 2 * NPART * sizeof(unsigned long long), c->stream) != cudaSuccess) {
    lbm_destroy(c);
    return LBM_ECUDA;
  }
  if (retile_default(c, 128) != LBM_OK) { lbm_destroy(c); return LBM_ECUDA; }
  *out = c;
  return LBM_OK;
}

}  // namespace

namespace pplbm {
Inst lbm_internal_inst(const lbm_ctx* c) { return c->hinst; }
unsigned long long lbm_internal_params_gen(const lbm_ctx* c) { return c->params_gen; }
}  // namespace pplbm

extern "C" {

void lbm_default_params(lbm_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->size = sizeof(lbm_params);
  p->geometry = LBM_GEOM_CHANNEL;
  p->thermal = 1;
  p->multiphase = 1;
  p->tau_f = 1.0;
  p->tau_g = 0.6;
  p->a = 2.0 / 49.0;
  p->b = 2.0 / 21.0;
  p->R = 1.0;
  p->omega = 0.32;
  p->beta = 1.16;
  p->c0 = 6.0;
  p->G = -1.0;
  p->T0_R = 0.9;
  p->Tin_R = 0.9;
  p->dTheat_R = 0.3;
  p->u_in = 0.01;
  p->rho_out = 5.95;
  p->rho_w = 5.95;
  p->G_wet = 9.0 * (1.0 + p->beta) * p->G;
  p->g_a = 5e-5;
  p->c_v = 6.0;
  p->heater_x0 = -1;
  p->heater_len = 5;
  p->heat_on_step = 10000;
  p->init_kind = LBM_INIT_UNIFORM;
  p->init_rho_in = 5.95;
  p->init_rho_out = 5.95;
  p->init_radius = 0.0;
  p->init_width = 2.0;
  p->perturb_amp = 0.0;
  p->seed = 0;
  p->rho_vapor = 3.2;
  p->source_model = LBM_SOURCE_GONG_CHENG;
  p->bubble_stats = 0;
}

size_t lbm_required_bytes(int32_t nx, int32_t ny, lbm_precision prec) {
  if (nx < 1 || ny < 1 || nx > kMaxDim || ny > kMaxDim) return 0;
  return make_layout(nx, ny, prec).total;
}

lbm_status lbm_create(lbm_ctx** out, int32_t nx, int32_t ny, lbm_precision prec, int32_t device, void* stream) {
  return create_impl(out, nx, ny, prec, device, stream, nullptr, 0);
}

lbm_status lbm_create_ex(lbm_ctx** out, int32_t nx, int32_t ny, lbm_precision prec, int32_t device, void* stream,
                         void* dev_buf, size_t dev_bytes) {
  if (!dev_buf) return LBM_EINVAL;
  return create_impl(out, nx, ny, prec, device, stream, dev_buf, dev_bytes);
}

lbm_status lbm_set_params(lbm_ctx* c, const lbm_params* p) {
  if (!c) return LBM_EINVAL;
  DeviceGuard g(c->device);
  lbm_status s = apply_params(c, p);
  if (s != LBM_OK) return s;
  if ((s = c->rows_default ? retile_default(c, c->cols) : set_tiling(c, c->cols, c->plan)) != LBM_OK) return s;
  InitSpec spec{};
  spec.kind = p->init_kind;
  spec.rho_in = p->init_rho_in;
  spec.rho_out = p->init_rho_out;
  spec.radius = p->init_radius;
  spec.width = p->init_width;
  spec.amp = p->perturb_amp;
  spec.T0 = c->hinst.T0;
  spec.seed = p->seed;
  spec.instance = 0;
  reset_state_mirror(c, 0, 1, 0.0);
  if ((s = upload_state(c)) != LBM_OK) return s;
  cudaError_t e = launch_init_builtin(c->prec == LBM_FP64, c->d_inst, c->nx, c->ny, spec, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
  ++c->launches;
  if ((s = launch(c, MODE_MOMENTS)) != LBM_OK) return s;
  return fetch_state(c);
}

lbm_status lbm_init_fields(lbm_ctx* c, const double* rho, const double* ux, const double* uy, const double* T,
                           size_t n) {
  NvtxRange nvtx("pplbm init_fields");
  if (!c || !rho || !ux || !uy) return fail(c, LBM_EINVAL, "NULL field");
  if (n != (size_t)c->nx * c->ny) return fail(c, LBM_EINVAL, "n != nx*ny");
  if (!c->have_params) return fail(c, LBM_ESTATE, "lbm_set_params first");
  DeviceGuard g(c->device);
  // host fields staged in the spare population buffer (buffer 1 is free at step 0)
  double* d_fields = reinterpret_cast<double*>(c->base + c->L.off_f[1]);
  LBM_CUDA(c, cudaMemcpyAsync(d_fields, rho, n * 8, cudaMemcpyHostToDevice, c->stream));
  LBM_CUDA(c, cudaMemcpyAsync(d_fields + n, ux, n * 8, cudaMemcpyHostToDevice, c->stream));
  LBM_CUDA(c, cudaMemcpyAsync(d_fields + 2 * n, uy, n * 8, cudaMemcpyHostToDevice, c->stream));
  if (T) LBM_CUDA(c, cudaMemcpyAsync(d_fields + 3 * n, T, n * 8, cudaMemcpyHostToDevice, c->stream));
  reset_state_mirror(c, 0, 1, 0.0);
  lbm_status s = upload_state(c);
  if (s != LBM_OK) return s;
  cudaError_t e = launch_init_from_fields(c->prec == LBM_FP64, c->d_inst, c->nx, c->ny, d_fields, T ? 1 : 0, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
  ++c->launches;
  // the buoyancy reference of step 0 (Eq. 14): the mean density of the initialised populations,
  // summed on the device (a host sum of the input field would hold the caller's thread for
  // milliseconds on large lattices)
  if ((s = launch(c, MODE_MOMENTS)) != LBM_OK) return s;
  c->step_host = 0;
  return fetch_state(c);
}

lbm_status lbm_step_async(lbm_ctx* c, int64_t nsteps) {
  NvtxRange nvtx("pplbm step");
  if (!c) return LBM_EINVAL;
  if (nsteps < 0) return fail(c, LBM_EINVAL, "nsteps < 0");
  if (!c->have_params) return fail(c, LBM_ESTATE, "lbm_set_params first");
  DeviceGuard g(c->device);
  if (nsteps >= 2 && use_persistent(c)) {
    const int kernel = step_kernel(c, c->cols);
    const bool full = needs_full_step(c->hinst);
    GridBar* bar = reinterpret_cast<GridBar*>(c->base + c->L.off_bar);
    FlowPlan flow{};
    if (overlapped(c)) {
      FlowInst& f = flow.single;
      f.tile_w = tile_cols(c->cols);
      f.strips = (c->nx + f.tile_w - 1) / f.tile_w;
      f.nbands = c->ntiles_step / f.strips;
      f.tall_rows = c->plan.tall_rows;
      f.tall_count = c->plan.tall_count;
      f.short_rows = c->plan.short_rows;
      f.n_open = c->nopen_step;
      f.perx = c->params.geometry != LBM_GEOM_CHANNEL;
      f.pery = c->params.geometry == LBM_GEOM_PERIODIC;
      flow.enabled = 1;
      flow.ninst = 1;
      flow.step0 = reinterpret_cast<long long*>(c->base + c->L.off_step0);
      flow.cell_done = reinterpret_cast<unsigned long long*>(c->base + c->L.off_cells);
    }
    for (int64_t done = 0; done < nsteps;) {
      const int n = (int)std::min<int64_t>(nsteps - done, 1 << 30);
      LBM_CUDA(c, cudaMemsetAsync(bar, 0, sizeof(GridBar), c->stream));
      if (flow.enabled)
        LBM_CUDA(c, cudaMemsetAsync(flow.cell_done, 0, (size_t)c->ntiles_step * sizeof(unsigned long long),
                                    c->stream));
      cudaError_t e = launch_persistent(c->prec == LBM_FP64, c->thermal, c->cols, kernel, full, c->d_inst,
                                        c->d_tiles_step, c->ntiles_step, n, bar, c->max_polls, c->stream, &c->hinst,
                                        flow);
      if (e != cudaSuccess) return cuda_fail(c, e, "persistent kernel launch");
      ++c->launches;
      done += n;
    }
    return LBM_OK;
  }
  for (int64_t k = 0; k < nsteps; ++k) {
    lbm_status s = launch(c, MODE_STEP);
    if (s != LBM_OK) return s;
  }
  return LBM_OK;
}

lbm_status lbm_sync(lbm_ctx* c) {
  NvtxRange nvtx("pplbm sync");
  if (!c) return LBM_EINVAL;
  DeviceGuard g(c->device);
  lbm_status s = fetch_state(c);
  if (s != LBM_OK) return s;
  if (c->h_state->status & STATUS_BOUNDS)
    return fail(c, LBM_EBOUNDS, std::to_string(c->h_state->bounds_hits) +
                                    " accesses outside their buffers were skipped (bounds-checked build)");
  if (c->h_state->status & STATUS_TIMEOUT)
    return fail(c, LBM_ETIMEOUT,
                "a bounded device wait gave up (a bulk tensor copy of the TMA step, or the grid barrier between the "
                "steps of a persistent launch); the lattice state is undefined until it is initialised again");
  if (c->h_state->status & STATUS_UNSTABLE)
    return fail(c, LBM_EUNSTABLE, "lattice left the EOS domain (rho <= 0, rho >= 1/b, NaN or psi radicand < 0)");
  return LBM_OK;
}

lbm_status lbm_step(lbm_ctx* c, int64_t nsteps) {
  lbm_status s = lbm_step_async(c, nsteps);
  if (s != LBM_OK) return s;
  return lbm_sync(c);
}

lbm_status lbm_read_fields(lbm_ctx* c, double* rho, double* ux, double* uy, double* T, size_t n) {
  NvtxRange nvtx("pplbm read_fields");
  if (!c) return LBM_EINVAL;
  if (n != (size_t)c->nx * c->ny) return fail(c, LBM_EINVAL, "n != nx*ny");
  if (!c->have_params) return fail(c, LBM_ESTATE, "lbm_set_params first");
  DeviceGuard g(c->device);
  lbm_status s = fetch_state(c);
  if (s != LBM_OK) return s;
  if ((s = launch(c, MODE_FIELDS)) != LBM_OK) return s;
  const double* d_out = reinterpret_cast<const double*>(c->base + c->L.off_f[(c->step_host + 1) & 1]);
  double* dst[4] = {rho, ux, uy, T};
  for (int k = 0; k < 4; ++k)
    if (dst[k]) LBM_CUDA(c, cudaMemcpyAsync(dst[k], d_out + k * n, n * 8, cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_get_populations(lbm_ctx* c, double* f, double* gout, size_t n) {
  if (!c || !f) return fail(c, LBM_EINVAL, "NULL f");
  if (n != 9 * (size_t)c->nx * c->ny) return fail(c, LBM_EINVAL, "n != 9*nx*ny");
  if (!c->have_params) return fail(c, LBM_ESTATE, "lbm_set_params first");
  DeviceGuard g(c->device);
  lbm_status s = fetch_state(c);
  if (s != LBM_OK) return s;
  if ((s = launch(c, MODE_POPS)) != LBM_OK) return s;
  const int spare = (int)((c->step_host + 1) & 1);
  const size_t elt = elt_size(c);
  std::vector<char> tmp(n * elt);
  const double rref[2] = {c->hinst.rho_ref, c->hinst.T_ref};
  double* outs[2] = {f, gout};
  const size_t offs[2] = {c->L.off_f[spare], c->L.off_g[spare]};
  for (int a = 0; a < 2; ++a) {
    if (!outs[a]) continue;
    if (a == 1 && !c->thermal) {
      for (int i = 0; i < 9; ++i) {
        const double w = i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
        for (size_t k = 0; k < (size_t)c->nx * c->ny; ++k) outs[a][i * (size_t)c->nx * c->ny + k] = w * c->hinst.T0;
      }
      continue;
    }
    LBM_CUDA(c, cudaMemcpy2DAsync(tmp.data(), c->nx * elt, c->base + offs[a], c->L.pitch * elt, c->nx * elt,
                                  9 * (size_t)c->ny, cudaMemcpyDeviceToHost, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
    const size_t np = (size_t)c->nx * c->ny;
    for (int i = 0; i < 9; ++i) {
      const double w = i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
      for (size_t k = 0; k < np; ++k) {
        const size_t idx = i * np + k;
        const double v = elt == 8 ? reinterpret_cast<const double*>(tmp.data())[idx]
                                  : (double)reinterpret_cast<const float*>(tmp.data())[idx];
        outs[a][idx] = v + w * rref[a];
      }
    }
  }
  return LBM_OK;
}

lbm_status lbm_set_populations(lbm_ctx* c, const double* f, const double* gin, size_t n, int64_t step,
                               double rho_avg_prev) {
  if (!c || !f) return fail(c, LBM_EINVAL, "NULL f");
  if (n != 9 * (size_t)c->nx * c->ny) return fail(c, LBM_EINVAL, "n != 9*nx*ny");
  if (step < 0) return fail(c, LBM_EINVAL, "step < 0");
  if (!c->have_params) return fail(c, LBM_ESTATE, "lbm_set_params first");
  DeviceGuard g(c->device);
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  const int buf = (int)(step & 1);
  const size_t elt = elt_size(c);
  const size_t np = (size_t)c->nx * c->ny;
  std::vector<char> tmp(n * elt);
  const double rref[2] = {c->hinst.rho_ref, c->hinst.T_ref};
  const double* ins[2] = {f, gin};
  const size_t offs[2] = {c->L.off_f[buf], c->L.off_g[buf]};
  for (int a = 0; a < 2; ++a) {
    for (int i = 0; i < 9; ++i) {
      const double w = i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
      for (size_t k = 0; k < np; ++k) {
        const size_t idx = i * np + k;
        const double full = ins[a] ? ins[a][idx] : w * c->hinst.T0;
        const double v = full - w * rref[a];
        if (elt == 8)
          reinterpret_cast<double*>(tmp.data())[idx] = v;
        else
          reinterpret_cast<float*>(tmp.data())[idx] = (float)v;
      }
    }
    LBM_CUDA(c, cudaMemcpy2DAsync(c->base + offs[a], c->L.pitch * elt, tmp.data(), c->nx * elt, c->nx * elt,
                                  9 * (size_t)c->ny, cudaMemcpyHostToDevice, c->stream));
    LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  const bool need_mean = std::isnan(rho_avg_prev);
  reset_state_mirror(c, step, 1, need_mean ? 0.0 : rho_avg_prev);
  lbm_status s = upload_state(c);
  if (s != LBM_OK) return s;
  // the moments pass also sets rho^(n-1) of the Hazi-Markus source to the injected density
  if ((need_mean || c->params.source_model == LBM_SOURCE_HAZI_MARKUS) && (s = launch(c, MODE_MOMENTS)) != LBM_OK)
    return s;
  if (!need_mean) {  // the moments pass overwrote the caller's mean: put it back
    reset_state_mirror(c, step, 1, rho_avg_prev);
    if ((s = upload_state(c)) != LBM_OK) return s;
  }
  return fetch_state(c);
}

lbm_status lbm_read_diagnostics(lbm_ctx* c, double* out, size_t n) {
  if (!c || !out) return fail(c, LBM_EINVAL, "NULL out");
  if (n < (size_t)LBM_D_COUNT) return fail(c, LBM_EINVAL, "n < LBM_D_COUNT");
  DeviceGuard g(c->device);
  lbm_status s = fetch_state(c);
  if (s != LBM_OK) return s;
  if (c->step_host <= 0) return fail(c, LBM_ESTATE, "no step taken yet");
  const long long last = c->step_host - 1;
  const double* rec = reinterpret_cast<const double*>(c->base + c->L.off_ring) + (last % RING) * NDIAG;
  LBM_CUDA(c, cudaMemcpyAsync(out, rec, NDIAG * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

namespace {
struct StateHeader {
  char magic[8];
  int32_t nx, ny, prec, abi;
  lbm_params params;
  InstState state;
};
}  // namespace

size_t lbm_state_bytes(const lbm_ctx* c) {
  if (!c) return 0;
  return sizeof(StateHeader) + (2 * 9 + 1) * (size_t)c->nx * c->ny * elt_size(c);
}

lbm_status lbm_save_state(lbm_ctx* c, void* host_buf, size_t bytes) {
  if (!c || !host_buf) return fail(c, LBM_EINVAL, "NULL buffer");
  if (bytes < lbm_state_bytes(c)) return fail(c, LBM_ENOMEM, "buffer smaller than lbm_state_bytes");
  if (!c->have_params) return fail(c, LBM_ESTATE, "lbm_set_params first");
  DeviceGuard g(c->device);
  lbm_status s = fetch_state(c);
  if (s != LBM_OK) return s;
  StateHeader h{};
  std::memcpy(h.magic, "PPLBMST", 8);
  h.nx = c->nx;
  h.ny = c->ny;
  h.prec = c->prec;
  h.abi = LBM_ABI_VERSION;
  h.params = c->params;
  h.state = *c->h_state;
  h.state.counter[0] = h.state.counter[1] = 0;
  char* dst = static_cast<char*>(host_buf);
  std::memcpy(dst, &h, sizeof(h));
  dst += sizeof(h);
  const size_t elt = elt_size(c);
  const int buf = (int)(c->step_host & 1);
  const size_t offs[2] = {c->L.off_f[buf], c->L.off_g[buf]};
  for (int a = 0; a < 2; ++a) {
    LBM_CUDA(c, cudaMemcpy2DAsync(dst, c->nx * elt, c->base + offs[a], c->L.pitch * elt, c->nx * elt,
                                  9 * (size_t)c->ny, cudaMemcpyDeviceToHost, c->stream));
    dst += 9 * (size_t)c->nx * c->ny * elt;
  }
  // rho^(n-1) of the Hazi-Markus source (kept in every state: resume is bitwise either way)
  LBM_CUDA(c, cudaMemcpy2DAsync(dst, c->nx * elt, c->base + c->L.off_rho_prev, c->L.pitch * elt, c->nx * elt,
                                (size_t)c->ny, cudaMemcpyDeviceToHost, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

lbm_status lbm_load_state(lbm_ctx* c, const void* host_buf, size_t bytes) {
  if (!c || !host_buf) return fail(c, LBM_EINVAL, "NULL buffer");
  if (bytes < lbm_state_bytes(c)) return fail(c, LBM_EINVAL, "buffer smaller than lbm_state_bytes");
  StateHeader h;
  std::memcpy(&h, host_buf, sizeof(h));
  if (std::memcmp(h.magic, "PPLBMST", 8) != 0 || h.nx != c->nx || h.ny != c->ny || h.prec != c->prec ||
      h.abi != LBM_ABI_VERSION)
    return fail(c, LBM_EINVAL, "state does not match this context");
  DeviceGuard g(c->device);
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  lbm_status s = apply_params(c, &h.params);
  if (s != LBM_OK) return s;
  if ((s = c->rows_default ? retile_default(c, c->cols) : set_tiling(c, c->cols, c->plan)) != LBM_OK) return s;
  *c->h_state = h.state;
  c->h_state->counter[0] = c->h_state->counter[1] = 0;
  if ((s = upload_state(c)) != LBM_OK) return s;
  const char* src = static_cast<const char*>(host_buf) + sizeof(h);
  const size_t elt = elt_size(c);
  const int buf = (int)(h.state.step & 1);
  const size_t offs[2] = {c->L.off_f[buf], c->L.off_g[buf]};
  for (int a = 0; a < 2; ++a) {
    LBM_CUDA(c, cudaMemcpy2DAsync(c->base + offs[a], c->L.pitch * elt, src, c->nx * elt, c->nx * elt,
                                  9 * (size_t)c->ny, cudaMemcpyHostToDevice, c->stream));
    src += 9 * (size_t)c->nx * c->ny * elt;
  }
  LBM_CUDA(c, cudaMemcpy2DAsync(c->base + c->L.off_rho_prev, c->L.pitch * elt, src, c->nx * elt, c->nx * elt,
                                (size_t)c->ny, cudaMemcpyHostToDevice, c->stream));
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  c->step_host = h.state.step;
  return LBM_OK;
}

lbm_status lbm_set_kernel(lbm_ctx* c, int32_t kernel) {
  if (!c) return LBM_EINVAL;
  if (kernel < LBM_KERNEL_AUTO || kernel > LBM_KERNEL_INTERIOR)
    return fail(c, LBM_EINVAL, "kernel must be LBM_KERNEL_AUTO, _SCALAR, _PAIRED, _TMA or _INTERIOR");
  c->kernel = kernel;
  if (!c->rows_default) return LBM_OK;
  DeviceGuard g(c->device);
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return retile_default(c, c->cols);
}

int32_t lbm_step_kernel(const lbm_ctx* c) { return c ? step_kernel(c, c->cols) : -1; }

lbm_status lbm_set_step_loop(lbm_ctx* c, int32_t loop) {
  if (!c) return LBM_EINVAL;
  if (loop < LBM_LOOP_AUTO || loop > LBM_LOOP_PERSISTENT)
    return fail(c, LBM_EINVAL, "loop must be LBM_LOOP_AUTO, _LAUNCHES or _PERSISTENT");
  c->loop = loop;
  return LBM_OK;
}

int32_t lbm_step_loop(lbm_ctx* c) {
  if (!c) return -1;
  if (!c->have_params) return c->loop == LBM_LOOP_PERSISTENT ? LBM_LOOP_PERSISTENT : LBM_LOOP_LAUNCHES;
  DeviceGuard g(c->device);
  if (!use_persistent(c)) return LBM_LOOP_LAUNCHES;
  return overlapped(c) ? LBM_LOOP_OVERLAPPED : LBM_LOOP_PERSISTENT;
}

lbm_status lbm_set_wait_limit(lbm_ctx* c, int64_t max_polls) {
  if (!c) return LBM_EINVAL;
  if (max_polls < 0 || max_polls > 0xffffffffll) return fail(c, LBM_EINVAL, "max_polls out of range");
  c->max_polls = (unsigned)max_polls;
  return LBM_OK;
}

lbm_status lbm_autotune(lbm_ctx* c, int32_t trial_steps, int32_t* cols_out, int32_t* rows_out) {
  if (!c || trial_steps < 1) return LBM_EINVAL;
  if (!c->have_params) return fail(c, LBM_ESTATE, "lbm_set_params first");
  DeviceGuard g(c->device);
  static const int kCols[] = {64, 128, 256};
  static const int kRows[] = {0, 4, 7, 10, 16, 24, 32, 48};
  cudaEvent_t e0, e1;
  LBM_CUDA(c, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(c, LBM_ECUDA, "cudaEventCreate");
  }
  float best = -1.0f;
  int best_c = 128, best_r = 0;
  lbm_status s = LBM_OK;
  for (int col : kCols) {
    for (int r : kRows) {
      if (r > c->ny) continue;
      if ((s = lbm_set_tiling(c, col, r)) != LBM_OK) break;
      if ((s = lbm_step_async(c, 2)) != LBM_OK) break;  // warm-up
      cudaEventRecord(e0, c->stream);
      if ((s = lbm_step_async(c, trial_steps)) != LBM_OK) break;
      cudaEventRecord(e1, c->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        s = fail(c, LBM_ECUDA, "autotune timing");
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (best < 0.0f || ms < best) {
        best = ms;
        best_c = col;
        best_r = r;
      }
    }
    if (s != LBM_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != LBM_OK) return s;
  if ((s = lbm_set_tiling(c, best_c, best_r)) != LBM_OK) return s;
  if (cols_out) *cols_out = best_c;
  if (rows_out) *rows_out = best_r;
  return lbm_sync(c);
}

lbm_status lbm_get_tiling(const lbm_ctx* c, int32_t* cols, int32_t* tall_rows, int32_t* tall_count,
                          int32_t* short_rows) {
  if (!c) return LBM_EINVAL;
  if (cols) *cols = c->cols;
  if (tall_rows) *tall_rows = c->plan.tall_rows;
  if (tall_count) *tall_count = c->plan.tall_count;
  if (short_rows) *short_rows = c->plan.short_rows;
  return LBM_OK;
}

lbm_status lbm_default_band_plan(int32_t nx, int32_t ny, int32_t cols, int64_t slots, int32_t* tall_rows,
                                 int32_t* tall_count, int32_t* short_rows) {
  if (nx < 1 || ny < 1 || !cols_supported(cols) || slots < 1) return LBM_EINVAL;
  const BandPlan p = default_band_plan(nx, ny, cols, slots);
  if (tall_rows) *tall_rows = p.tall_rows;
  if (tall_count) *tall_count = p.tall_count;
  if (short_rows) *short_rows = p.short_rows;
  return LBM_OK;
}

lbm_status lbm_set_tiling(lbm_ctx* c, int32_t cols, int32_t rows) {
  if (!c) return LBM_EINVAL;
  if (cols == 0) cols = 128;
  if (!cols_supported(cols)) return fail(c, LBM_EINVAL, "cols must be 64, 128 or 256");
  if (rows < 0) return fail(c, LBM_EINVAL, "rows must be >= 0");
  DeviceGuard g(c->device);
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  if (rows == 0) return retile_default(c, cols);
  rows = std::min(rows, c->ny);
  if (rows < kMinRows && rows < c->ny) return fail(c, LBM_EINVAL, "rows must be >= 4 (or the full height)");
  const lbm_status s = set_tiling(c, cols, BandPlan{0, 0, rows});
  if (s == LBM_OK) c->rows_default = false;
  return s;
}

lbm_status lbm_read_diagnostics_range(lbm_ctx* c, int64_t first, int64_t count, double* out) {
  if (!c) return LBM_EINVAL;
  if (count < 0 || (count > 0 && !out)) return fail(c, LBM_EINVAL, "count < 0 or NULL out");
  DeviceGuard g(c->device);
  lbm_status s = fetch_state(c);
  if (s != LBM_OK) return s;
  if (count == 0) return LBM_OK;
  const long long oldest = std::max<long long>(0, c->step_host - RING);
  if (first < oldest || first + count > c->step_host)
    return fail(c, LBM_EINVAL, "requested steps are not in the diagnostics ring");
  const double* ring = reinterpret_cast<const double*>(c->base + c->L.off_ring);
  long long done = 0;
  while (done < count) {  // at most two contiguous pieces of the ring
    const long long slot = (first + done) % RING;
    const long long n = std::min<long long>(count - done, RING - slot);
    LBM_CUDA(c, cudaMemcpyAsync(out + done * NDIAG, ring + slot * NDIAG, (size_t)n * NDIAG * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
    done += n;
  }
  LBM_CUDA(c, cudaStreamSynchronize(c->stream));
  return LBM_OK;
}

int64_t lbm_get_step(const lbm_ctx* c) { return c ? c->step_host : -1; }
int64_t lbm_launch_count(const lbm_ctx* c) { return c ? c->launches : -1; }
void* lbm_get_stream(const lbm_ctx* c) { return c ? static_cast<void*>(c->stream) : nullptr; }

double lbm_critical_temperature(const lbm_params* p) {
  if (!p) return NAN;
  return 0.0778 * p->a / (0.45724 * p->b * p->R);
}

lbm_status lbm_destroy(lbm_ctx* c) {
  if (!c) return LBM_OK;
  {
    DeviceGuard g(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->own_mem && c->base) cudaFree(c->base);
    if (c->h_state) cudaFreeHost(c->h_state);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  }
  delete c;
  return LBM_OK;
}

const char* lbm_status_string(lbm_status s) {
  switch (s) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "out of memory";
    case LBM_EUNSTABLE: return "lattice unstable";
    case LBM_ETIMEOUT: return "device wait timed out";
    case LBM_ECUDA: return "CUDA error";
    case LBM_EBUDGET: return "memory budget exceeded";
    case LBM_ESTATE: return "call out of order";
    case LBM_EBOUNDS: return "index outside its buffer (bounds-checked build)";
  }
  return "unknown status";
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

}  // extern "C"
