// Internal host/device descriptors of the pplbm library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>  // header-only: ranges cost nothing unless a profiler is attached
#include <stdint.h>

#include "pplbm.h"

namespace pplbm {

// An NVTX range around a host call (step, chunk, readback), named for the profiler's timeline.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Per-tile partial sums folded by the last CTA of an instance:
// mass, energy, T summed over the heater-adjacent row, inlet flux, outlet flux.
constexpr int NPART = 9;  // mass, energy, heater row T, inflow, outflow, vapour area, wall / heater / zone vapour
// The tiles of a launch add their partial sums into NPART signed 64-bit fixed-point totals;
// total j has 52 - ceil(log2(m_j)) fraction bits, m_j the most nodes that feed it (nx ny for
// mass, energy and the vapour counts, nx for the heater row, ny for the inlet and outlet
// columns).  Every per-node term is at most 1024 in magnitude, so a total stays below 2^62,
// and integer addition is exact and commutative, so the totals do not depend on the order in
// which tiles finish.
constexpr int FIX_BITS = 52;
constexpr int NDIAG = 12;  // LBM_D_COUNT
constexpr int RING = 1024;  // diagnostics records kept per instance

enum : int { GEOM_PERIODIC = 0, GEOM_CHANNEL = 1, GEOM_WALLS = 2, GEOM_POOL = 3 };
enum : int { MODE_STEP = 0, MODE_FIELDS = 1, MODE_POPS = 2, MODE_MOMENTS = 3 };
enum : unsigned { STATUS_UNSTABLE = 1u, STATUS_TIMEOUT = 2u, STATUS_BOUNDS = 4u };

// Device-resident mutable state of one lattice instance.
// Step n uses the slots n & 1 of counter and p_probe and the slot n % 4 of the open-end mass
// exchange: the overlapped persistent loop has tiles of two consecutive steps in flight.
struct InstState {
  long long step;       // steps completed
  int local_read;       // 1: buffer (step & 1) holds post-stream populations (after init/load)
  unsigned int status;  // sticky STATUS_* bits, cleared by the host
  unsigned int counter[2];   // tiles of step n that have posted their partials, in slot n & 1
  unsigned int bounds_hits;  // accesses a bounds-checked build rejected (STATUS_BOUNDS), else 0
  unsigned int open_posted[4];  // open-end tiles of step n that posted open_mass, in slot n % 4
  int pad0;
  double rho_avg[2];    // domain-mean rho of step n in slot n & 1 (buoyancy of step n+1, Eq. 14)
  double p_probe[4];    // EOS pressure at (1, ny/2) and (nx-2, ny/2) of step n in slots 2 (n & 1) + {0, 1}
  long long open_mass[4];  // fixed-point mass that step n's pull took in and let out through the
                           // open ends (created minus lost populations), in slot n % 4
};

// Read-only description of one lattice instance (host-filled, device-resident).
struct Inst {
  int nx, ny, pitch, geometry;
  long long plane;      // elements per population plane (pitch * ny)
  void* f[2];           // population double buffer: 9 planes each (storage precision)
  void* g[2];
  int multiphase, pad1;
  double omega_f, omega_g;          // 1/tau_f, 1/tau_g
  double a, b, R, kappa, sqrtTc, inv_sqrtTc;
  double psi_scale;                 // 2/(c0 G) of Eq. 11
  double beta, G2, Ghalf;           // Eq. 8 beta; Eq. 10 g1 = 2G, g2 = G/2
  double Gwet_psiw;                 // G_wet * psi(rho_w, T0) of Eq. 15
  double g_a, inv_cv;
  double T0, T_in, T_heat, u_in, rho_out;
  double rho_ref, T_ref;            // storage offsets: f stored as f - w_i rho_ref, g as g - w_i T_ref
  double alpha0;                    // alpha(T0) of Eq. 12 for isothermal runs
  // FP32 reference state of the pseudopotential: psi is carried as psi - psi_ref,
  // evaluated from exact difference forms of Eq. 12 in rho - rho_ref and T - T_ref
  double psi_ref, rad_ref, p_ref, inv_u1r, inv_Dr, sa_r, sqrtT_r, rr2_Dr;
  int heater_x0, heater_len;
  long long heat_on_step;
  double rho_vapor;                 // vapour threshold of the bubble diagnostics
  int source_model, bubble_stats;   // 0 Gong-Cheng, 1 Hazi-Markus (first Eq. 19); count vapour nodes
  void* rho_prev;                   // rho^(n-1) - rho_ref per node (storage precision, pitch layout)
  const void* tmaps;                // FP32: 4 tensor maps of 128 bytes (f of buffers 0, 1, then g); or null
  InstState* st;
  unsigned long long* sums;         // NPART fixed-point totals of the current launch (zero between launches)
  double fix_scale[NPART];          // 2^f_j, f_j the fraction bits of total j
  double fix_unscale[NPART];        // 2^-f_j
  double* ring;                     // RING records of NDIAG doubles
  // Element offsets within a population buffer: population i of node n sits at n + poff[i]
  // (poff[i] = i * plane), and on a node with no wall or open-end link it is pulled from
  // n + loff[i] (the node n - c_i, in plane i: loff[i] = poff[i] - c_iy pitch - c_ix).
  int loff[9], poff[9];
  // Derived constants of the step, formed on the host only (so that every kernel converts the
  // same doubles): (1 - beta)/2 of Eq. 8; the outlet density, inlet and heater temperatures as
  // deviations from the storage references; the vapour threshold as a density deviation; and
  // the reference parts of Eqs. 9 and 15 on a row next to the bottom wall, wall0 + d wall1 with
  // d = psi - psi_ref (its fluid neighbours have sum G_i c_iy = 3G and its solid neighbours
  // sum w_i c_iy = -1/6; the two parts cancel exactly for a balanced wall, which keeps the FP32
  // force free of the cancellation).
  double mix, drho_out, dT_in, dT_heat, drho_vapor, wall0, wall1;
  // products of constants of the FP32 equation of state, formed on the host: R / (1 - b rho_ref),
  // a / D(rho_ref) with D(rho) = 1 + 2 b rho - (b rho)^2, 2 b rho_ref, -kappa / sqrt(Tc),
  // a rho_ref^2 / D(rho_ref)
  double R_u1r, a_Dr, twob_rr, nk_sTc, a_rr2_Dr;
};

// State of the grid-wide barrier between the steps of a persistent launch (device memory,
// zeroed by the host before every persistent launch).  count: CTAs arrived at the current
// barrier; gen: barriers completed; status: 1 once a CTA gave up waiting; next[2]: the
// dynamic tile counters of even and odd steps.
//
// Overlapped form (FlowPlan.enabled, a parameter of the launch; a lattice or a batch whose
// tiling has more tiles than resident CTAs): the CTAs draw (step, tile) tickets in order from
// `claim`, and a tile of step s waits only for what it reads, instead of a barrier for all the
// tiles: the tiles of its instance around it to have finished step s - 1 (cell_done), step
// s - 2 of its instance to be complete (its mean density), and the instance's open-end tiles
// of step s - 1 to have posted the mass that crossed the inlet and outlet; its buoyancy mean is
// the mean of step s - 2 plus that mass over the nodes (Eq. 14).  Tiles of two consecutive
// steps run at once, so the end of one step overlaps the start of the next.
struct FlowInst {  // one instance's tiling
  int strips, nbands, tile_w;             // tiles per band, bands per step, output columns per tile
  int tall_rows, tall_count, short_rows;  // band layout (row y -> band)
  int n_open;                             // tiles per step with an open end
  int perx, pery;                         // strips wrap in x (walls, periodic), bands in y (periodic)
  int pad;
  long long cell_base;                    // the instance's first tile position in cell_done
};
struct FlowPlan {
  int enabled;
  int ninst;
  FlowInst single;                 // the instance of a single-lattice launch (inst == nullptr)
  const FlowInst* inst;            // a batch's table (device memory), indexed by Tile.inst
  long long* step0;                // per instance: its step when the launch starts (written by the
                                   // launch's first CTA before the tickets start)
  unsigned long long* cell_done;   // per tile position (cell_base + band * strips + strip): steps
                                   // of this launch it has finished (zeroed before the launch)
};
struct GridBar {
  unsigned int count, gen, status, pad;
  unsigned int next[2];
  unsigned long long claim;  // overlapped form: (step, tile) tickets drawn in this launch
};
// Bounded waits of the persistent launch: a CTA stops waiting at a barrier after wait_ns
// nanoseconds of polling, or after max_polls polls when max_polls > 0 (a test lowers it to
// make the wait run out while the other CTAs are still busy).
constexpr unsigned long long BARRIER_WAIT_NS = 5000000000ull;

// One CTA's work: output columns [x0, x0 + W) of instance `inst`, rows [y0, y1).
struct Tile {
  int inst, x0, y0, y1;
  int local;   // index of this tile among its instance's tiles (partials slot)
  int ntiles;  // tiles of this instance in the launch
  int interior;  // 1: every column the tile pulls, [x0 - 2, x0 + cols - 6), lies in [1, nx - 2] of a
                 // channel or walls lattice (no open end, no wrap): the interior path may take it
  int open_end;  // 1: the tile's output columns include the inlet or the outlet of a channel
};
// Whether a tile of a cols-thread step tiling starting at column x0 may take the interior path.
inline int tile_is_interior(int geometry, int nx, int cols, int x0) {
  return (geometry == GEOM_CHANNEL || geometry == GEOM_WALLS) && x0 - 2 >= 1 && x0 + (cols - 8) + 1 <= nx - 2;
}
// Tiles that take the general loop (dispatched before the interior tiles of their class).
inline bool general_tile(const Tile& t) { return !t.interior; }

// Launchers (defined per precision).  Tiles must have been built for `cols`.
// kernel: a resolved form (resolve_kernel): LBM_KERNEL_SCALAR, _INTERIOR, _PAIRED or _TMA.
// full: the instances use the pool geometry, the Hazi-Markus source or bubble statistics, which
// only the step's full form handles (the lean form leaves them out of the hot loop).
// h_inst: host copy of the launch's only instance (the lean scalar step then takes its
// constants as a kernel parameter), or null for launches over several instances.
// max_polls: poll cap of the TMA form's row waits (0: its full limit; lbm_set_wait_limit).
cudaError_t launch_lbm(int fp64, int thermal, int cols, int mode, int kernel, bool full, const Inst* d_inst,
                       const Tile* d_tiles, int ntiles, cudaStream_t s, const Inst* h_inst = nullptr,
                       unsigned max_polls = 0);
// nsteps steps of the step kernel in one cooperative launch (tiles drawn dynamically from a
// counter, a bounded grid barrier between steps; MODE_STEP only).  grid <= resident CTAs of
// the device; bar: zeroed GridBar in device memory.
// flow.enabled: the overlapped form (one instance; more tiles than resident CTAs).
cudaError_t launch_persistent(int fp64, int thermal, int cols, int kernel, bool full, const Inst* d_inst,
                              const Tile* d_tiles, int ntiles, int nsteps, GridBar* bar, unsigned max_polls,
                              cudaStream_t s, const Inst* h_inst, const FlowPlan& flow);
// CTAs one persistent launch may hold on the current device (SMs x resident CTAs per SM).
long long persistent_slots(int fp64, int thermal, int cols, int kernel, bool full, bool single);
// Whether an instance needs the step's full form.
inline bool needs_full_step(const Inst& I) {
  return I.geometry == GEOM_POOL || I.source_model != 0 || I.bubble_stats != 0;
}
// The step-kernel form a launch takes for a requested LBM_KERNEL_* value.  LBM_KERNEL_AUTO
// and LBM_KERNEL_INTERIOR take the one-column kernel with its interior path (tiles away from
// open ends and wraps run a loop without any per-node boundary logic; the others run the
// general loop), the fastest form on GB300, whenever the step's lean form applies, else the
// plain one-column kernel.  FP64 has no other forms; the paired kernel has no Hazi-Markus
// source; the TMA kernel needs 128-column tiles, the step's lean form and the instances'
// tensor maps (tmaps: all instances of the launch have them).
constexpr int TMA_TILE_COLS = 128;
inline int resolve_kernel(int requested, int fp64, bool full, bool hazi, bool tmaps, int cols) {
  if (requested == LBM_KERNEL_AUTO || requested == LBM_KERNEL_INTERIOR)
    return full ? LBM_KERNEL_SCALAR : LBM_KERNEL_INTERIOR;
  if (fp64) return LBM_KERNEL_SCALAR;
  if (requested == LBM_KERNEL_PAIRED) return hazi ? LBM_KERNEL_SCALAR : LBM_KERNEL_PAIRED;
  if (requested == LBM_KERNEL_TMA && !full && tmaps && cols == TMA_TILE_COLS) return LBM_KERNEL_TMA;
  return LBM_KERNEL_SCALAR;
}
// f = f^eq(rho,u), g = g^eq(T,u) into buffer 0 from 4 planes of nx*ny doubles (rho, ux, uy, T).
cudaError_t launch_init_from_fields(int fp64, const Inst* d_inst, int nx, int ny, const double* d_fields,
                                    int has_T, cudaStream_t s);
// Built-in initial state (uniform or seeded disk) into buffer 0.
struct InitSpec {
  int kind;
  double rho_in, rho_out, radius, width, amp, T0;
  unsigned long long seed;
  int instance;
};
cudaError_t launch_init_builtin(int fp64, const Inst* d_inst, int nx, int ny, InitSpec spec, cudaStream_t s);

bool cols_supported(int cols);

// Host helpers shared by the context API and the allocation-free step.
// check_params: nullptr when p is valid for an nx x ny lattice, else the reason.
const char* check_params(int nx, int ny, const lbm_params* p);
// fill_inst: the physics part of an instance descriptor (buffer and scratch pointers
// are left null); nullptr on success, else the reason.
const char* fill_inst(Inst& I, const lbm_params* p, int nx, int ny, int pitch, long long plane, int fp64);
// Rows per band of the default tiling for CTAs of `cols` threads.
// Rows per band of a cols-wide step tiling of an nx x ny lattice: the band height
// that covers the lattice in the fewest row-iterations per CTA slot, counting the 4
// halo rows (plus about one row of fixed cost) every band adds, the `slots` CTAs one
// wave holds and half a tile of tail.  Never below 4 rows unless the lattice is lower.
int default_band_rows(int nx, int ny, int cols, long long slots);
// Rows of a step tiling, per strip of cols - 8 columns: tall_count bands of tall_rows from the
// bottom, then bands of short_rows (the last one possibly lower) up to the top; every strip's
// tall bands are dispatched before any short band (uniform tilings: tall_count = 0).
struct BandPlan {
  int tall_rows, tall_count, short_rows;
};
// The default step tiling of an nx x ny lattice for `slots` CTA slots: the uniform band height
// of default_band_rows, or, where the same cost model finds it cheaper, tall bands of 2h rows
// followed by about one wave of short bands of h rows, which the block scheduler dispatches
// last, so the end of the step is filled by short tiles while most rows pay the halo of tall
// bands only.
BandPlan default_band_plan(int nx, int ny, int cols, long long slots);
// CTAs of the step kernel (storage precision, thermal flag, tile columns, kernel
// form) that one wave of the current device holds: SMs x resident CTAs per SM.
long long step_wave_slots(int fp64, int thermal, int cols, int kernel);
int resident_ctas_f32(int thermal, int cols, int kernel);
int resident_ctas_f64(int thermal, int cols, int kernel);
// The instance descriptor of a context (device pointers included), for batching.
Inst lbm_internal_inst(const lbm_ctx* c);
// Changes whenever the context's descriptor is rewritten (parameters or a loaded state).
unsigned long long lbm_internal_params_gen(const lbm_ctx* c);

}  // namespace pplbm
