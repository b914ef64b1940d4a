/*
 * Oracle: plain FP64 CPU restatement of the pseudopotential thermal lattice
 * Boltzmann step of Mukherjee, Basu & Mondal (arXiv 2009.05264), Sec. 2.
 *
 * TEST INFRASTRUCTURE ONLY -- loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the library.  Every step below is
 * written node by node in the order the method defines, with no blocking,
 * fusion or reordering:
 *   1. moments            rho = sum f (Eq. 4), u_eq = sum f c / rho (Eq. 6), T = sum g (Eq. 17)
 *   2. equation of state  Peng-Robinson p(rho, T) (Eq. 12), psi (Eq. 11), (dp/dT)_rho
 *   3. body force         Shan-Chen (Eqs. 9-10), wetting (Eq. 15), buoyancy (Eq. 14)
 *   4. velocities         du = F/rho (Eq. 5), u_act = u_eq + F/(2 rho) (Eq. 7)
 *   5. f collision        BGK (Eq. 2) toward f^eq (Eq. 3) plus exact-difference forcing (Eq. 5)
 *   6. g collision        BGK toward g^eq(T, u_act) (Eq. 18) plus source phi (second Eq. 19, or the
 *                         first with rho^n - rho^(n-1) for its temporal density gradient)
 *   7. diagnostics        mass, energy, domain-mean density for the next step's buoyancy;
 *                         vapour area, its footprint on the bottom wall and over the heater,
 *                         and the vapour in the columns around the heater
 *   8. streaming (Eqs. 1, 16) and the boundary conditions of Sec. 2.C: halfway
 *      bounce-back walls, anti-bounce-back wall/heater/inlet temperature,
 *      non-equilibrium bounce-back (Zou-He) velocity inlet and pressure outlet,
 *      zero-gradient temperature outlet.
 *
 * Readings of passages that are garbled or silent (all follow the same list
 * as the CUDA library's documentation):
 *   Eq. 6 is read with the division by rho; Eq. 7 with F dt/(2 rho) (the tau_f
 *   factor is 1 at tau_f = 1); Eq. 9 with psi(x1) and psi^2(x1) inside the sums;
 *   Eq. 10 with g1 = 2G, g2 = G/2 (so g1 = 4 g2 and sum G_i c_ix^2 = c0 G);
 *   alpha(T) of Eq. 12 with sqrt(T/Tc); Eq. 14 as F_y = -(rho - rho_avg) g_a with
 *   rho_avg the previous step's mean; Eq. 15 with D2Q9 weights w_i and
 *   psi_w = psi(rho_w, T0); Eq. 16 with the relaxation term -(g - g^eq)/tau_g;
 *   the second Eq. 19 (Gong-Cheng source) is the one used.  Sec. 2.C fixes no
 *   discretisation of div u in that source nor of the outlet's zero temperature
 *   gradient: div u is taken by central differences, except that on a row next to
 *   a wall the wall-normal derivative is the one-sided difference over the two
 *   fluid rows; the outlet node takes all nine post-stream g of the node upstream.
 *   (With u = 0 at the solid site instead, a row-alternating u_y mode grows at the
 *   walls, and with only the unknown g copied the outlet diverges, both within
 *   about 10^4 steps.)
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* The per-node loops over rows may run on several threads (orc_set_threads, in a build with
 * OpenMP; without it the pragmas are ignored).  Every node's arithmetic is the same either
 * way and every sum over nodes stays serial in row-major order, so the results do not depend
 * on the thread count.  The default is one thread (no thread pool is started). */
#define ORC_ROWS _Pragma("omp parallel for if(L->threads > 1) num_threads(L->threads > 1 ? L->threads : 1)")
#define ORC_ROWS_STATUS \
  _Pragma("omp parallel for reduction(max : status) if(L->threads > 1) num_threads(L->threads > 1 ? L->threads : 1)")

/* D2Q9 velocity set (Fig. 1) with the standard weights 4/9, 1/9, 1/36. */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double WT[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double CS2 = 1.0 / 3.0; /* lattice sound speed squared, c_s = c / sqrt(3) */

struct orc_lattice {
  int nx, ny;
  double* f; /* post-stream f^n */
  double* g; /* post-stream g^n */
  double rho_avg_prev;
  double* rho_prev; /* rho^(n-1) per node (the Hazi-Markus source's time derivative) */
  int64_t step;
  double diag[ORC_D_COUNT];
  /* per-node work arrays of one step */
  double *rho, *ux, *uy, *T, *psi, *dpdT, *Fx, *Fy, *uax, *uay, *phi;
  double *fpost, *gpost, *fnew, *gnew;
  unsigned char* unknown;
  int threads; /* threads of the per-node loops (<= 1: serial) */
};

static size_t nodes(const orc_lattice* L) { return (size_t)L->nx * (size_t)L->ny; }
static size_t nid(const orc_lattice* L, int x, int y) { return (size_t)y * L->nx + x; }
static size_t pid(const orc_lattice* L, int i, int x, int y) {
  return ((size_t)i * L->ny + y) * L->nx + x;
}
static int wrap(int v, int n) { return ((v % n) + n) % n; }

orc_lattice* orc_create(int32_t nx, int32_t ny) {
  if (nx < 1 || ny < 1) return NULL;
  orc_lattice* L = (orc_lattice*)calloc(1, sizeof(orc_lattice));
  if (!L) return NULL;
  L->nx = nx;
  L->ny = ny;
  size_t n = nodes(L);
  L->f = calloc(9 * n, sizeof(double));
  L->g = calloc(9 * n, sizeof(double));
  L->fpost = calloc(9 * n, sizeof(double));
  L->gpost = calloc(9 * n, sizeof(double));
  L->fnew = calloc(9 * n, sizeof(double));
  L->gnew = calloc(9 * n, sizeof(double));
  L->unknown = calloc(9 * n, 1);
  double** scalars[] = {&L->rho, &L->ux, &L->uy, &L->T, &L->psi, &L->dpdT,
                        &L->Fx,  &L->Fy, &L->uax, &L->uay, &L->phi, &L->rho_prev};
  int ok = L->f && L->g && L->fpost && L->gpost && L->fnew && L->gnew && L->unknown;
  for (size_t k = 0; k < sizeof(scalars) / sizeof(scalars[0]); ++k) {
    *scalars[k] = calloc(n, sizeof(double));
    ok = ok && *scalars[k];
  }
  if (!ok) {
    orc_destroy(L);
    return NULL;
  }
  return L;
}

int orc_set_threads(orc_lattice* L, int threads) {
  if (!L || threads < 1) return ORC_BAD_ARG;
  L->threads = threads;
  return ORC_OK;
}

void orc_destroy(orc_lattice* L) {
  if (!L) return;
  free(L->f); free(L->g); free(L->fpost); free(L->gpost); free(L->fnew); free(L->gnew);
  free(L->unknown);
  free(L->rho); free(L->ux); free(L->uy); free(L->T); free(L->psi); free(L->dpdT);
  free(L->Fx); free(L->Fy); free(L->uax); free(L->uay); free(L->phi); free(L->rho_prev);
  free(L);
}

/* ---------------------------------------------------------------------------
 * Equation of state, Eq. 12 and the definitions that follow it.
 * ------------------------------------------------------------------------- */

/* a = 0.45724 R^2 Tc^2 / pc and b = 0.0778 R Tc / pc give Tc = 0.0778 a / (0.45724 b R). */
double orc_Tc(const orc_params* P) { return 0.0778 * P->a / (0.45724 * P->b * P->R); }

static double pr_kappa(const orc_params* P) {
  return 0.37464 + 1.54226 * P->omega - 0.26992 * P->omega * P->omega;
}

/* alpha(T) = [1 + kappa (1 - sqrt(T/Tc))]^2 */
static double pr_alpha(const orc_params* P, double T) {
  double s = 1.0 + pr_kappa(P) * (1.0 - sqrt(T / orc_Tc(P)));
  return s * s;
}

double orc_pressure(const orc_params* P, double rho, double T) {
  double a = P->a, b = P->b;
  return rho * P->R * T / (1.0 - b * rho) -
         a * pr_alpha(P, T) * rho * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho);
}

/* (dp/dT) at constant rho: d(alpha)/dT = -kappa sqrt(alpha) / sqrt(T Tc). */
double orc_dpdT(const orc_params* P, double rho, double T) {
  double a = P->a, b = P->b, Tc = orc_Tc(P);
  double dalpha = -pr_kappa(P) * sqrt(pr_alpha(P, T)) / sqrt(T * Tc);
  return rho * P->R / (1.0 - b * rho) - a * dalpha * rho * rho / (1.0 + 2.0 * b * rho - b * b * rho * rho);
}

/* Eq. 11: psi = sqrt(2 (p - c_s^2 rho) / (c0 g)).  NaN when the radicand is negative. */
double orc_psi(const orc_params* P, double rho, double T) {
  double rad = 2.0 * (orc_pressure(P, rho, T) - CS2 * rho) / (P->c0 * P->G);
  if (!(rad >= 0.0)) return NAN;
  return sqrt(rad);
}

/* Pressure and (dp/dT)_rho of the fluid being simulated: Peng-Robinson in the
 * two-phase model, the lattice ideal gas p = c_s^2 rho in single-phase runs. */
static double fluid_pressure(const orc_params* P, double rho, double T) {
  return P->multiphase ? orc_pressure(P, rho, T) : CS2 * rho;
}
static double fluid_dpdT(const orc_params* P, double rho, double T) {
  return P->multiphase ? orc_dpdT(P, rho, T) : 0.0;
}

/* ---------------------------------------------------------------------------
 * Maxwell equal-area construction on Eq. 12 (coexistence densities, Sec. 2.D).
 * ------------------------------------------------------------------------- */

static double maxwell_area(const orc_params* P, double T, double rv, double rl, double ps) {
  /* integral over v = 1/rho of (p - p_sat) dv, written in rho: int (p - ps)/rho^2 drho */
  const int n = 20000; /* Simpson, even number of intervals */
  double h = (rl - rv) / n, s = 0.0;
  for (int k = 0; k <= n; ++k) {
    double r = rv + k * h;
    double w = (k == 0 || k == n) ? 1.0 : (k % 2 ? 4.0 : 2.0);
    s += w * (orc_pressure(P, r, T) - ps) / (r * r);
  }
  return s * h / 3.0;
}

static double bisect_root(const orc_params* P, double T, double ps, double lo, double hi) {
  /* root of p(rho) - ps on [lo, hi] where the sign changes */
  double flo = orc_pressure(P, lo, T) - ps;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    double fm = orc_pressure(P, mid, T) - ps;
    if ((fm > 0) == (flo > 0)) {
      lo = mid;
      flo = fm;
    } else {
      hi = mid;
    }
  }
  return 0.5 * (lo + hi);
}

int orc_maxwell(const orc_params* P, double T, double* rho_v, double* rho_l, double* p_sat) {
  double rmax = 1.0 / P->b;
  const int n = 200000;
  /* spinodal densities: the local maximum then the local minimum of p(rho) */
  double r_a = -1, r_b = -1, prev = orc_pressure(P, rmax * 1e-7, T);
  int rising = 1;
  for (int k = 2; k < n; ++k) {
    double r = rmax * k / n;
    double p = orc_pressure(P, r, T);
    if (rising && p < prev) {
      r_a = rmax * (k - 1) / n;
      rising = 0;
    } else if (!rising && p > prev) {
      r_b = rmax * (k - 1) / n;
      break;
    }
    prev = p;
  }
  if (r_a < 0 || r_b < 0) return ORC_BAD_ARG; /* supercritical: no loop */
  double p_hi = orc_pressure(P, r_a, T);
  double p_lo = orc_pressure(P, r_b, T);
  if (p_lo < 1e-14) p_lo = 1e-14;
  double rv = 0, rl = 0, ps = 0;
  for (int it = 0; it < 200; ++it) {
    ps = 0.5 * (p_lo + p_hi);
    rv = bisect_root(P, T, ps, rmax * 1e-9, r_a);
    rl = bisect_root(P, T, ps, r_b, rmax * (1.0 - 1e-12));
    double area = maxwell_area(P, T, rv, rl, ps);
    if (area > 0)
      p_lo = ps;
    else
      p_hi = ps;
  }
  *rho_v = rv;
  *rho_l = rl;
  *p_sat = ps;
  return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Equilibria, Eqs. 3 and 18.
 * ------------------------------------------------------------------------- */

static double equilibrium(int i, double m, double ux, double uy) {
  double cu = CX[i] * ux + CY[i] * uy;
  double uu = ux * ux + uy * uy;
  return WT[i] * m * (1.0 + cu / CS2 + 0.5 * cu * cu / (CS2 * CS2) - 0.5 * uu / CS2);
}

/* ---------------------------------------------------------------------------
 * Lattice sites.  site() maps a lattice site to the fluid node whose values it
 * carries, or reports a solid node.  Channel walls are the rows y = -1 and
 * y = ny; the open ends carry zero-gradient ghost columns x = -1 and x = nx
 * that repeat the first and last fluid column.  The pool's open top carries a
 * zero-gradient ghost row y = ny that repeats row ny - 1.
 * ------------------------------------------------------------------------- */
static int site(const orc_lattice* L, const orc_params* P, int x, int y, size_t* idx) {
  if (P->geometry == ORC_PERIODIC) {
    x = wrap(x, L->nx);
    y = wrap(y, L->ny);
  } else {
    if (P->geometry == ORC_POOL && y >= L->ny) y = L->ny - 1;
    if (y < 0 || y >= L->ny) return 0;
    if (P->geometry == ORC_WALLS || P->geometry == ORC_POOL) {
      x = wrap(x, L->nx);
    } else {
      if (x < 0) x = 0;
      if (x >= L->nx) x = L->nx - 1;
    }
  }
  *idx = nid(L, x, y);
  return 1;
}

static int heater_on(const orc_params* P, int64_t step) {
  return P->thermal && P->heater_len > 0 && step >= P->heat_on_step;
}

/* Wall temperature at solid site (sx, sy): the bottom-wall heater segment is
 * superheated once switched on; every other wall point is at T_in. */
static double wall_T(const orc_lattice* L, const orc_params* P, int sx, int sy, int64_t step) {
  double Tc = orc_Tc(P);
  if (P->geometry == ORC_WALLS || P->geometry == ORC_POOL) sx = wrap(sx, L->nx);
  if (sy < 0 && heater_on(P, step) && sx >= P->heater_x0 && sx < P->heater_x0 + P->heater_len)
    return (P->Tin_R + P->dTheat_R) * Tc;
  return P->Tin_R * Tc;
}

static int finite_ok(double v) { return isfinite(v); }

/* ---------------------------------------------------------------------------
 * One step's macroscopic stage: moments, EOS, forces, velocities.
 * ------------------------------------------------------------------------- */
static int macroscopic(orc_lattice* L, const orc_params* P) {
  const int nx = L->nx, ny = L->ny;
  const size_t n = nodes(L);
  const double Tc = orc_Tc(P), T0 = P->T0_R * Tc;
  int status = ORC_OK;

  /* Moments, Eqs. 4, 6, 17 */
  ORC_ROWS_STATUS
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t k = nid(L, x, y);
      double rho = 0, jx = 0, jy = 0, T = 0;
      for (int i = 0; i < 9; ++i) {
        double fi = L->f[pid(L, i, x, y)];
        rho += fi;
        jx += fi * CX[i];
        jy += fi * CY[i];
      }
      if (P->thermal) {
        for (int i = 0; i < 9; ++i) T += L->g[pid(L, i, x, y)];
      } else {
        T = T0;
      }
      L->rho[k] = rho;
      L->ux[k] = jx / rho;
      L->uy[k] = jy / rho;
      L->T[k] = T;
      if (!(rho > 0.0) || !finite_ok(rho) || !finite_ok(T)) status = ORC_UNSTABLE;
      if (P->multiphase && rho * P->b >= 1.0) status = ORC_UNSTABLE;
    }
  if (status != ORC_OK) return status;

  /* Pseudopotential (Eqs. 11-12) and (dp/dT)_rho */
  ORC_ROWS_STATUS
  for (size_t k = 0; k < n; ++k) {
    if (P->multiphase) {
      L->psi[k] = orc_psi(P, L->rho[k], L->T[k]);
      if (!finite_ok(L->psi[k])) status = ORC_UNSTABLE;
    }
    L->dpdT[k] = fluid_dpdT(P, L->rho[k], L->T[k]);
  }
  if (status != ORC_OK) return status;
  const double psi_w = P->multiphase ? orc_psi(P, P->rho_w, T0) : 0.0;

  /* Body force: Shan-Chen (Eqs. 9-10), wetting (Eq. 15), buoyancy (Eq. 14) */
  ORC_ROWS
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t k = nid(L, x, y);
      double Fx = 0, Fy = 0;
      if (P->multiphase) {
        double s1x = 0, s1y = 0, s2x = 0, s2y = 0, swx = 0, swy = 0;
        for (int i = 1; i < 9; ++i) {
          double Gi = (i <= 4) ? 2.0 * P->G : 0.5 * P->G; /* g1 = 4 g2 */
          size_t m;
          if (site(L, P, x + CX[i], y + CY[i], &m)) {
            s1x += Gi * L->psi[m] * CX[i];
            s1y += Gi * L->psi[m] * CY[i];
            s2x += Gi * L->psi[m] * L->psi[m] * CX[i];
            s2y += Gi * L->psi[m] * L->psi[m] * CY[i];
          } else {
            swx += WT[i] * psi_w * CX[i];
            swy += WT[i] * psi_w * CY[i];
          }
        }
        Fx = -P->beta * L->psi[k] * s1x - 0.5 * (1.0 - P->beta) * s2x;
        Fy = -P->beta * L->psi[k] * s1y - 0.5 * (1.0 - P->beta) * s2y;
        Fx += -P->G_wet * L->psi[k] * swx;
        Fy += -P->G_wet * L->psi[k] * swy;
      }
      Fy += -(L->rho[k] - L->rho_avg_prev) * P->g_a; /* gravity along -y */
      L->Fx[k] = Fx;
      L->Fy[k] = Fy;
      /* Eq. 7: actual velocity */
      L->uax[k] = L->ux[k] + Fx / (2.0 * L->rho[k]);
      L->uay[k] = L->uy[k] + Fy / (2.0 * L->rho[k]);
    }
  return status;
}

/* Velocity u_act at lattice site (x, y): zero at solid sites, the ghost copy at open ends. */
static void uact_at(const orc_lattice* L, const orc_params* P, int x, int y, double* ux, double* uy) {
  size_t m;
  if (site(L, P, x, y, &m)) {
    *ux = L->uax[m];
    *uy = L->uay[m];
  } else {
    *ux = 0.0;
    *uy = 0.0;
  }
}

/* Solve the dense system A z = rhs (n <= 3) by Gaussian elimination with partial pivoting. */
static void solve_small(int n, double A[3][3], double* rhs, double* z) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
    if (piv != c) {
      for (int k = 0; k < n; ++k) {
        double t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t;
      }
      double t = rhs[c]; rhs[c] = rhs[piv]; rhs[piv] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      double m = A[r][c] / A[c][c];
      for (int k = c; k < n; ++k) A[r][k] -= m * A[c][k];
      rhs[r] -= m * rhs[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = rhs[r];
    for (int k = r + 1; k < n; ++k) s -= A[r][k] * z[k];
    z[r] = s / A[r][r];
  }
}

/* Velocity inlet at x = 0 (Zou-He non-equilibrium bounce-back, Sec. 2.C):
 * impose u = (u_in, 0) on the populations that streaming left unknown. */
static void inlet_node(orc_lattice* L, const orc_params* P, int y) {
  const int x = 0;
  const double u = P->u_in;
  int U[3], nu = 0;
  double Kr = 0, Kx = 0, Ky = 0;
  for (int i = 0; i < 9; ++i) {
    if (L->unknown[pid(L, i, x, y)]) {
      U[nu++] = i;
    } else {
      double fi = L->fnew[pid(L, i, x, y)];
      Kr += fi;
      Kx += fi * CX[i];
      Ky += fi * CY[i];
    }
  }
  if (nu == 3) {
    /* the three unknowns all have c_x = +1: sum f = rho and sum f c_x = rho u give rho */
    double rho = (Kr - Kx) / (1.0 - u);
    /* non-equilibrium bounce-back normal to the inlet: f1 - f1eq = f3 - f3eq */
    double f1 = L->fnew[pid(L, 3, x, y)] + equilibrium(1, rho, u, 0.0) - equilibrium(3, rho, u, 0.0);
    /* remaining two from sum f c_x = rho u and sum f c_y = 0 */
    double f5 = 0.5 * (rho * u - Kx - f1 - Ky);
    double f8 = 0.5 * (rho * u - Kx - f1 + Ky);
    L->fnew[pid(L, 1, x, y)] = f1;
    L->fnew[pid(L, 5, x, y)] = f5;
    L->fnew[pid(L, 8, x, y)] = f8;
  } else if (nu == 2) {
    /* corner: unknowns rho, f_a, f_b from the three moment conditions */
    int a = U[0], b = U[1];
    double A[3][3] = {{-1.0, 1.0, 1.0}, {-u, (double)CX[a], (double)CX[b]}, {0.0, (double)CY[a], (double)CY[b]}};
    double rhs[3] = {-Kr, -Kx, -Ky}, z[3];
    solve_small(3, A, rhs, z);
    L->fnew[pid(L, a, x, y)] = z[1];
    L->fnew[pid(L, b, x, y)] = z[2];
  }
  if (P->thermal) {
    /* anti-bounce-back: inlet temperature T_in */
    double Tin = P->Tin_R * orc_Tc(P);
    for (int k = 0; k < nu; ++k) {
      int i = U[k];
      L->gnew[pid(L, i, x, y)] = -L->gpost[pid(L, OPP[i], x, y)] + 2.0 * WT[i] * Tin;
    }
  }
}

/* Pressure outlet at x = nx-1 (Zou-He): impose rho = rho_out, u_y = 0. */
static void outlet_node(orc_lattice* L, const orc_params* P, int y) {
  const int x = L->nx - 1;
  const double rho = P->rho_out;
  int U[3], nu = 0;
  double Kr = 0, Kx = 0, Ky = 0;
  for (int i = 0; i < 9; ++i) {
    if (L->unknown[pid(L, i, x, y)]) {
      U[nu++] = i;
    } else {
      double fi = L->fnew[pid(L, i, x, y)];
      Kr += fi;
      Kx += fi * CX[i];
      Ky += fi * CY[i];
    }
  }
  if (nu == 3) {
    /* the unknowns all have c_x = -1: sum f = rho and sum f c_x = rho u give u */
    double u = (Kx - (rho - Kr)) / rho;
    double f3 = L->fnew[pid(L, 1, x, y)] - (equilibrium(1, rho, u, 0.0) - equilibrium(3, rho, u, 0.0));
    /* remaining two from sum f c_x = rho u and sum f c_y = 0 */
    double f6 = 0.5 * (Kx - rho * u - f3 - Ky);
    double f7 = 0.5 * (Kx - rho * u - f3 + Ky);
    L->fnew[pid(L, 3, x, y)] = f3;
    L->fnew[pid(L, 6, x, y)] = f6;
    L->fnew[pid(L, 7, x, y)] = f7;
  } else if (nu == 2) {
    /* corner: sum f = rho_out and sum f c_y = 0 fix the two unknowns */
    int a = U[0], b = U[1];
    double A[3][3] = {{1.0, 1.0, 0.0}, {(double)CY[a], (double)CY[b], 0.0}, {0, 0, 1.0}};
    double rhs[3] = {rho - Kr, -Ky, 0.0}, z[3];
    solve_small(2, A, rhs, z);
    L->fnew[pid(L, a, x, y)] = z[0];
    L->fnew[pid(L, b, x, y)] = z[1];
  }
  if (P->thermal) {
    /* zero temperature gradient: the outlet node takes all post-stream populations
     * of the node one upstream (their wall links already applied) */
    for (int i = 0; i < 9; ++i) L->gnew[pid(L, i, x, y)] = L->gnew[pid(L, i, x - 1, y)];
  }
}

/* Pool top y = ny-1 (free surface of Sec. 2.D, a constant-pressure boundary): Zou-He
 * with rho = rho_out and u_x = 0 for the three populations streaming would bring from
 * above (c_y = -1), and zero temperature gradient (all nine g of the row below). */
static void top_node(orc_lattice* L, const orc_params* P, int x) {
  const int y = L->ny - 1;
  const double rho = P->rho_out;
  double Kr = 0, Ky = 0, Kx = 0;
  for (int i = 0; i < 9; ++i) {
    if (CY[i] == -1) continue;
    double fi = L->fnew[pid(L, i, x, y)];
    Kr += fi;
    Kx += fi * CX[i];
    Ky += fi * CY[i];
  }
  /* unknowns 4, 7, 8 carry c_y = -1: sum f = rho and sum f c_y = rho u_y give u_y */
  double u = (Ky - (rho - Kr)) / rho;
  double f4 = L->fnew[pid(L, 2, x, y)] - (equilibrium(2, rho, 0.0, u) - equilibrium(4, rho, 0.0, u));
  /* remaining two from sum f c_y = rho u_y and sum f c_x = 0 */
  double f7 = 0.5 * (Ky - rho * u - f4 + Kx); /* c_7 = (-1, -1) */
  double f8 = 0.5 * (Ky - rho * u - f4 - Kx); /* c_8 = (1, -1) */
  L->fnew[pid(L, 4, x, y)] = f4;
  L->fnew[pid(L, 7, x, y)] = f7;
  L->fnew[pid(L, 8, x, y)] = f8;
  if (P->thermal)
    for (int i = 0; i < 9; ++i) L->gnew[pid(L, i, x, y)] = L->gnew[pid(L, i, x, y - 1)];
}

static int one_step(orc_lattice* L, const orc_params* P) {
  const int nx = L->nx, ny = L->ny;
  const size_t n = nodes(L);
  int status = macroscopic(L, P);
  if (status != ORC_OK) return status;

  /* f collision: Eqs. 1-3 with the exact-difference force term of Eq. 5 */
  ORC_ROWS
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t k = nid(L, x, y);
      double rho = L->rho[k];
      double dux = L->Fx[k] / rho, duy = L->Fy[k] / rho;
      for (int i = 0; i < 9; ++i) {
        double fi = L->f[pid(L, i, x, y)];
        double feq = equilibrium(i, rho, L->ux[k], L->uy[k]);
        double feq_shift = equilibrium(i, rho, L->ux[k] + dux, L->uy[k] + duy);
        L->fpost[pid(L, i, x, y)] = fi - (fi - feq) / P->tau_f + (feq_shift - feq);
      }
    }

  /* g collision: Eq. 16 with g^eq of Eq. 18 and the source of the second Eq. 19 */
  double source_total = 0.0;
  if (P->thermal) {
    ORC_ROWS
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        size_t k = nid(L, x, y);
        double uxp, uyp, uxm, uym, t;
        uact_at(L, P, x + 1, y, &uxp, &t);
        uact_at(L, P, x - 1, y, &uxm, &t);
        uact_at(L, P, x, y + 1, &t, &uyp);
        uact_at(L, P, x, y - 1, &t, &uym);
        /* second-order central differences; on a row next to a wall the wall-normal
         * derivative is the one-sided difference over the two fluid rows */
        double dyu = 0.5 * (uyp - uym);
        const int wall_row = P->geometry != ORC_PERIODIC &&
                             (y == 0 || (y == ny - 1 && P->geometry != ORC_POOL)); /* pool top: open */
        if (wall_row) {
          double uyc;
          uact_at(L, P, x, y, &t, &uyc);
          if (ny == 1 && P->geometry != ORC_POOL) dyu = 0.0;
          else if (y == 0) dyu = uyp - uyc;
          else dyu = uyc - uym;
        }
        double divu = 0.5 * (uxp - uxm) + dyu;
        double T = L->T[k];
        double phi;
        if (P->source_model == 1) {
          /* first Eq. 19 (Hazi-Markus): T/(rho^2 c_v) (dp/dT)_rho drho/dt + T div u, the
           * temporal density gradient by the two-level difference rho^n - rho^(n-1) */
          double rho = L->rho[k];
          phi = T / (rho * rho * P->c_v) * L->dpdT[k] * (rho - L->rho_prev[k]) + T * divu;
        } else {
          phi = T * (1.0 - L->dpdT[k] / (L->rho[k] * P->c_v)) * divu;
        }
        L->phi[k] = phi;
        for (int i = 0; i < 9; ++i) {
          double gi = L->g[pid(L, i, x, y)];
          double geq = equilibrium(i, T, L->uax[k], L->uay[k]);
          L->gpost[pid(L, i, x, y)] = gi - (gi - geq) / P->tau_g + WT[i] * phi;
        }
      }
    for (size_t k = 0; k < n; ++k) source_total += L->phi[k];
  }

  /* Diagnostics of this step (row-major FP64 sums) */
  double mass = 0, energy = 0;
  for (size_t k = 0; k < n; ++k) {
    mass += L->rho[k];
    energy += L->T[k];
  }
  double dp = 0, dtstar = 0, flux_in = 0, flux_out = 0;
  if (P->geometry == ORC_CHANNEL && nx >= 3) {
    size_t a = nid(L, 1, ny / 2), b = nid(L, nx - 2, ny / 2);
    dp = fluid_pressure(P, L->rho[a], L->T[a]) - fluid_pressure(P, L->rho[b], L->T[b]);
    for (int y = 0; y < ny; ++y) {
      size_t i0 = nid(L, 0, y), i1 = nid(L, nx - 1, y);
      flux_in += L->rho[i0] * L->uax[i0];
      flux_out += L->rho[i1] * L->uax[i1];
    }
  }
  if (heater_on(P, L->step) && P->geometry != ORC_PERIODIC) {
    double Tc = orc_Tc(P), Tw = (P->Tin_R + P->dTheat_R) * Tc, Tnb = 0;
    int cnt = 0;
    for (int x = P->heater_x0; x < P->heater_x0 + P->heater_len && x < nx; ++x) {
      if (x < 0) continue;
      Tnb += L->T[nid(L, x, 0)];
      ++cnt;
    }
    if (cnt > 0) {
      Tnb /= cnt;
      double Tbulk = energy / (double)n;
      dtstar = (Tw - Tnb) / (Tw - Tbulk);
    }
  }
  L->diag[ORC_D_STEP] = (double)L->step;
  L->diag[ORC_D_MASS] = mass;
  L->diag[ORC_D_ENERGY] = energy;
  L->diag[ORC_D_RHO_AVG] = mass / (double)n;
  L->diag[ORC_D_DP] = dp;
  L->diag[ORC_D_DTSTAR] = dtstar;
  L->diag[ORC_D_FLUX_IN] = flux_in;
  L->diag[ORC_D_FLUX_OUT] = flux_out;
  L->diag[ORC_D_SOURCE] = source_total;
  /* Bubble diagnostics (vapour: rho below rho_vapor), from this step's moments */
  double area = 0, wall = 0, heat = 0, zone = 0;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      if (!(L->rho[nid(L, x, y)] < P->rho_vapor)) continue;
      area += 1.0;
      if (x >= P->heater_x0 - P->heater_len && x < P->heater_x0 + 2 * P->heater_len) zone += 1.0;
      if (y == 0 && P->geometry != ORC_PERIODIC) {
        wall += 1.0;
        if (x >= P->heater_x0 && x < P->heater_x0 + P->heater_len) heat += 1.0;
      }
    }
  L->diag[ORC_D_VAPOR_AREA] = area;
  L->diag[ORC_D_WALL_VAPOR] = wall;
  L->diag[ORC_D_HEATER_VAPOR] = heat;
  L->diag[ORC_D_ZONE_VAPOR] = zone;
  memcpy(L->rho_prev, L->rho, n * sizeof(double)); /* rho^n becomes the next step's rho^(n-1) */

  /* Streaming (Eqs. 1, 16) with the wall rules; open-end unknowns marked */
  memset(L->unknown, 0, 9 * n);
  for (int i = 0; i < 9; ++i) {
    ORC_ROWS
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        int sx = x - CX[i], sy = y - CY[i];
        size_t dst = pid(L, i, x, y);
        if (P->geometry == ORC_PERIODIC) {
          sx = wrap(sx, nx);
          sy = wrap(sy, ny);
        } else if (P->geometry == ORC_POOL && sy >= ny) {
          L->unknown[dst] = 1; /* link from above the open top: set by top_node */
          continue;
        } else if (sy < 0 || sy >= ny) {
          /* link from a wall row: halfway bounce-back for f, anti-bounce-back for g */
          L->fnew[dst] = L->fpost[pid(L, OPP[i], x, y)];
          if (P->thermal)
            L->gnew[dst] = -L->gpost[pid(L, OPP[i], x, y)] + 2.0 * WT[i] * wall_T(L, P, sx, sy, L->step);
          continue;
        } else if (P->geometry == ORC_WALLS || P->geometry == ORC_POOL) {
          sx = wrap(sx, nx);
        } else if (sx < 0 || sx >= nx) {
          L->unknown[dst] = 1; /* set by the inlet/outlet conditions below */
          continue;
        }
        L->fnew[dst] = L->fpost[pid(L, i, sx, sy)];
        if (P->thermal) L->gnew[dst] = L->gpost[pid(L, i, sx, sy)];
      }
  }
  if (P->geometry == ORC_CHANNEL) {
    for (int y = 0; y < ny; ++y) inlet_node(L, P, y);
    for (int y = 0; y < ny; ++y) outlet_node(L, P, y);
  }
  if (P->geometry == ORC_POOL)
    for (int x = 0; x < nx; ++x) top_node(L, P, x);

  double* t = L->f; L->f = L->fnew; L->fnew = t;
  t = L->g; L->g = L->gnew; L->gnew = t;
  L->rho_avg_prev = mass / (double)n;
  L->step += 1;
  return ORC_OK;
}

static int check_geometry(const orc_lattice* L, const orc_params* P) {
  if (P->geometry == ORC_CHANNEL && (L->nx < 3 || L->ny < 2)) return ORC_BAD_ARG;
  if (P->geometry == ORC_WALLS && L->ny < 2) return ORC_BAD_ARG;
  if (P->geometry == ORC_POOL && L->ny < 3) return ORC_BAD_ARG;
  if (P->geometry < 0 || P->geometry > 3) return ORC_BAD_ARG;
  return ORC_OK;
}

int orc_step(orc_lattice* L, const orc_params* P, int64_t nsteps) {
  if (!L || !P || nsteps < 0) return ORC_BAD_ARG;
  if (check_geometry(L, P) != ORC_OK) return ORC_BAD_ARG;
  for (int64_t s = 0; s < nsteps; ++s) {
    int st = one_step(L, P);
    if (st != ORC_OK) return st;
  }
  return ORC_OK;
}

int orc_init_fields(orc_lattice* L, const orc_params* P, const double* rho, const double* ux,
                    const double* uy, const double* T) {
  if (!L || !P || !rho || !ux || !uy) return ORC_BAD_ARG;
  const size_t n = nodes(L);
  double mass = 0;
  for (int y = 0; y < L->ny; ++y)
    for (int x = 0; x < L->nx; ++x) {
      size_t k = nid(L, x, y);
      for (int i = 0; i < 9; ++i) {
        L->f[pid(L, i, x, y)] = equilibrium(i, rho[k], ux[k], uy[k]);
        L->g[pid(L, i, x, y)] = T ? equilibrium(i, T[k], ux[k], uy[k]) : 0.0;
      }
      mass += rho[k];
    }
  L->rho_avg_prev = mass / (double)n;
  memcpy(L->rho_prev, rho, n * sizeof(double)); /* no density change before the first step */
  L->step = 0;
  memset(L->diag, 0, sizeof(L->diag));
  return ORC_OK;
}

int orc_set_populations(orc_lattice* L, const double* f, const double* g, int64_t step,
                        double rho_avg_prev) {
  if (!L || !f) return ORC_BAD_ARG;
  const size_t n = nodes(L);
  memcpy(L->f, f, 9 * n * sizeof(double));
  if (g) memcpy(L->g, g, 9 * n * sizeof(double));
  L->step = step;
  L->rho_avg_prev = rho_avg_prev;
  for (size_t k = 0; k < n; ++k) { /* injected state: no density change before its first step */
    double r = 0.0;
    for (int i = 0; i < 9; ++i) r += L->f[(size_t)i * n + k];
    L->rho_prev[k] = r;
  }
  return ORC_OK;
}

int orc_get_populations(const orc_lattice* L, double* f, double* g) {
  if (!L) return ORC_BAD_ARG;
  const size_t n = nodes(L);
  if (f) memcpy(f, L->f, 9 * n * sizeof(double));
  if (g) memcpy(g, L->g, 9 * n * sizeof(double));
  return ORC_OK;
}

int64_t orc_get_step(const orc_lattice* L) { return L ? L->step : -1; }
double orc_get_rho_avg_prev(const orc_lattice* L) { return L ? L->rho_avg_prev : NAN; }

int orc_fields(orc_lattice* L, const orc_params* P, double* rho, double* ux, double* uy,
               double* T, double* Fx, double* Fy) {
  if (!L || !P) return ORC_BAD_ARG;
  if (check_geometry(L, P) != ORC_OK) return ORC_BAD_ARG;
  int st = macroscopic(L, P);
  const size_t n = nodes(L);
  for (size_t k = 0; k < n; ++k) {
    if (rho) rho[k] = L->rho[k];
    if (ux) ux[k] = L->uax[k];
    if (uy) uy[k] = L->uay[k];
    if (T) T[k] = L->T[k];
    if (Fx) Fx[k] = L->Fx[k];
    if (Fy) Fy[k] = L->Fy[k];
  }
  return st;
}

int orc_last_diag(const orc_lattice* L, double* out) {
  if (!L || !out) return ORC_BAD_ARG;
  memcpy(out, L->diag, sizeof(L->diag));
  return ORC_OK;
}
