/*
 * Oracle for the pseudopotential thermal lattice Boltzmann flow-boiling step of
 * Mukherjee, Basu & Mondal, "Mesoscopic Characterization of Bubble Dynamics in
 * Flow Boiling following A Pseudopotential-based Approach" (arXiv 2009.05264).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded FP64 CPU
 * restatement of Sec. 2 (Eqs. 1-19) and the boundary conditions of Sec. 2.C.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
 * load it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Lattice: D2Q9, velocities c_i in the order
 *   0 (0,0) 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1) 5 (1,1) 6 (-1,1) 7 (-1,-1) 8 (1,-1)
 * Populations are stored as 9 planes of ny rows of nx doubles, index
 * (i*ny + y)*nx + x.  The state is the post-stream (pre-collision) f^n, g^n.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_PERIODIC = 0, ORC_CHANNEL = 1, ORC_WALLS = 2,
       ORC_POOL = 3 /* pool boiling (Sec. 2.D): periodic x, bottom wall, pressure top (rho_out) */ };

enum {
  ORC_OK = 0,
  ORC_BAD_ARG = 1,
  ORC_UNSTABLE = 3 /* rho <= 0, rho >= 1/b, NaN, or psi radicand >= 0 */
};

typedef struct orc_params {
  int32_t geometry;   /* ORC_PERIODIC, ORC_CHANNEL (inlet/outlet + walls), ORC_WALLS (walls, periodic x),
                         ORC_POOL (bottom wall, periodic x, constant-pressure top) */
  int32_t thermal;    /* 1: evolve g (Eq. 16); 0: T frozen at T0 */
  int32_t multiphase; /* 1: Shan-Chen + wetting forces (Eqs. 9, 15); 0: single-phase, p = rho/3 */
  double tau_f, tau_g;
  double a, b, R, omega, beta, c0, G; /* Eq. 12 a, b, R, omega; Eq. 8 beta; Eq. 11 c0 and g (here G) */
  double T0_R, Tin_R, dTheat_R;        /* reduced temperatures T/T_c (Eq. 13) */
  double u_in, rho_out, rho_w, G_wet, g_a, c_v;
  int32_t heater_x0, heater_len;
  int64_t heat_on_step;
  double rho_vapor;   /* density below which a node counts as vapour (bubble diagnostics) */
  int32_t source_model; /* energy source: 0 = Gong-Cheng (second Eq. 19), 1 = Hazi-Markus (first Eq. 19) */
  int32_t reserved0;
} orc_params;

/* Diagnostics of one step, computed from that step's moments. */
enum {
  ORC_D_STEP = 0, ORC_D_MASS, ORC_D_ENERGY, ORC_D_RHO_AVG, ORC_D_DP, ORC_D_DTSTAR,
  ORC_D_FLUX_IN, ORC_D_FLUX_OUT, ORC_D_SOURCE,
  ORC_D_VAPOR_AREA,   /* nodes with rho < rho_vapor (bubble area, lattice units) */
  ORC_D_WALL_VAPOR,   /* of those, nodes on the row next to the bottom wall (vapour footprint) */
  ORC_D_HEATER_VAPOR, /* of those, nodes above heater sites x_h <= x < x_h + n_h */
  ORC_D_ZONE_VAPOR,   /* vapour nodes in the columns x_h - n_h <= x < x_h + 2 n_h (the bubble at the heater) */
  ORC_D_COUNT
};

typedef struct orc_lattice orc_lattice;

orc_lattice* orc_create(int32_t nx, int32_t ny);
void orc_destroy(orc_lattice* L);
/* Threads for the per-node loops (a build with OpenMP; otherwise ignored).  Results do not
 * depend on it: node arithmetic is unchanged and every sum over nodes stays serial.
 * Default 1.  ORC_BAD_ARG for threads < 1. */
int orc_set_threads(orc_lattice* L, int threads);

/* f = f^eq(rho, u) (Eq. 3), g = g^eq(T, u) (Eq. 18); step = 0; rho_avg of the
 * previous step is taken as the mean of the initial rho.  Arrays: ny*nx row-major. */
int orc_init_fields(orc_lattice* L, const orc_params* P, const double* rho, const double* ux,
                    const double* uy, const double* T);
/* Post-stream populations f^n, g^n (9*ny*nx each; g ignored when NULL). */
int orc_set_populations(orc_lattice* L, const double* f, const double* g, int64_t step,
                        double rho_avg_prev);
int orc_get_populations(const orc_lattice* L, double* f, double* g);
int64_t orc_get_step(const orc_lattice* L);
double orc_get_rho_avg_prev(const orc_lattice* L);

/* Advance nsteps time steps.  Returns ORC_OK or ORC_UNSTABLE. */
int orc_step(orc_lattice* L, const orc_params* P, int64_t nsteps);

/* Macroscopic fields of the current state: rho (Eq. 4), actual velocity (Eq. 7),
 * T (Eq. 17) and total body force F.  Any output pointer may be NULL. */
int orc_fields(orc_lattice* L, const orc_params* P, double* rho, double* ux, double* uy,
               double* T, double* Fx, double* Fy);

/* Diagnostics of the most recent step (ORC_D_COUNT doubles). */
int orc_last_diag(const orc_lattice* L, double* out);

/* Equation of state (Eq. 12), its temperature derivative and the
 * pseudopotential (Eq. 11); T is an absolute lattice temperature. */
double orc_Tc(const orc_params* P);
double orc_pressure(const orc_params* P, double rho, double T);
double orc_dpdT(const orc_params* P, double rho, double T);
double orc_psi(const orc_params* P, double rho, double T);

/* Maxwell equal-area coexistence densities at absolute temperature T. */
int orc_maxwell(const orc_params* P, double T, double* rho_v, double* rho_l, double* p_sat);

#ifdef __cplusplus
}
#endif
#endif
