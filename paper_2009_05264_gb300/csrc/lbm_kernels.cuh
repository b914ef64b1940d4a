// Fused D2Q9 pseudopotential thermal LB step for sm_103a.
//
// One kernel does a whole time step of Mukherjee, Basu & Mondal (arXiv
// 2009.05264, Sec. 2): pull-streaming with the Sec. 2.C boundary conditions,
// moments (Eqs. 4, 6, 17), Peng-Robinson EOS and pseudopotential (Eqs. 11-12),
// Shan-Chen + wetting + buoyancy force (Eqs. 9, 10, 14, 15), actual velocity
// (Eq. 7), BGK + exact-difference collision of f (Eqs. 2, 3, 5), Gong-Cheng
// source and collision of g (Eqs. 16, 18, second Eq. 19), and FP64 partial
// sums of the step's diagnostics folded by the last CTA.
//
// Data layout: populations are structure-of-arrays, 9 planes of ny rows of
// `pitch` elements, double-buffered; the kernel reads the post-collision
// populations of step n-1 (or, right after initialisation, post-stream ones)
// from buffer (n & 1) and writes post-collision populations of step n to
// buffer ((n + 1) & 1).  In FP32 the stored values are deviations from the
// rest-state weights, f_i - w_i rho_ref and g_i - w_i T_ref, which keeps the
// low-order bits for the small non-equilibrium parts.
//
// Work decomposition: a CTA owns W output columns [x0, x0 + W) and a band of
// rows [y0, y1), and marches up the band one row per iteration.  The force at
// a node needs psi on its 8 neighbours, and the divergence of u_act in the g
// source needs u_act (hence the force) on the 4 neighbours, so psi is needed
// two nodes out.  Each CTA therefore keeps three-row rings in shared memory
// of psi and u_act over W + 4 columns; W threads own the output columns and 4
// lanes of a fifth warp compute the 2-column halos on each side.  At iteration
// k the CTA pulls row r = y0 - 2 + k, computes force, u_act and the f
// collision of row r - 1, and the g collision of row r - 2.  Populations are
// read once per CTA (plus the halo columns and 4 rows per band), all loads and
// stores of a warp are to consecutive addresses.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "lbm_internal.h"

namespace pplbm {

__host__ __device__ constexpr int lat_cx(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int lat_cy(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int lat_opp(int i) {
  return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
}
template <typename Real>
__host__ __device__ constexpr Real lat_w(int i) {
  return i == 0 ? Real(4.0 / 9.0) : (i <= 4 ? Real(1.0 / 9.0) : Real(1.0 / 36.0));
}

__device__ __forceinline__ int wrap_index(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

__device__ __forceinline__ float ld_ro(const float* p) { return __ldg(p); }
__device__ __forceinline__ double ld_ro(const double* p) { return __ldg(p); }

template <int BLOCK>
__device__ __forceinline__ void block_sum(double (&v)[NPART], double (*red)[NPART]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < NPART; ++j) {
    double x = v[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp][j] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < NPART; ++j) {
      double s = 0.0;
      for (int w = 0; w < BLOCK / 32; ++w) s += red[w][j];
      v[j] = s;
    }
  }
}

// ---------------------------------------------------------------------------
// The fused kernel.  MODE_STEP advances one step; MODE_FIELDS writes rho, u_act
// and T (FP64) of the current state to the spare f buffer; MODE_POPS writes
// the post-stream populations to the spare buffers; MODE_MOMENTS only folds
// the mean density into the buoyancy slot of the previous step.
// ---------------------------------------------------------------------------
template <typename Real, bool THERMAL, int W, int MODE>
__global__ void __launch_bounds__(W + 32, (sizeof(Real) == 4 ? (W <= 64 ? 6 : (W <= 128 ? 3 : 2))
                                                              : (W <= 64 ? 4 : (W <= 128 ? 2 : 1))))
lbm_fused_kernel(const Inst* __restrict__ insts, const Tile* __restrict__ tiles) {
  constexpr int BLOCK = W + 32;
  constexpr int NS = W + 4;
  __shared__ Inst sI;
  __shared__ Real sPsi[3][NS];
  __shared__ Real sUx[3][NS];
  __shared__ Real sUy[3][NS];
  __shared__ Real sG[THERMAL ? 3 : 1][9][THERMAL ? W : 1];
  __shared__ double sRed[BLOCK / 32][NPART];
  __shared__ int sLast;

  const int tid = threadIdx.x;
  const Tile tile = tiles[blockIdx.x];
  {
    const int* src = reinterpret_cast<const int*>(insts + tile.inst);
    int* dst = reinterpret_cast<int*>(&sI);
    for (int k = tid; k < (int)(sizeof(Inst) / 4); k += BLOCK) dst[k] = src[k];
  }
  __syncthreads();

  const int nx = sI.nx, ny = sI.ny, pitch = sI.pitch;
  const long long plane = sI.plane;
  InstState* st = sI.st;
  const long long step = st->step;
  const bool local = st->local_read != 0;
  const bool perx = sI.geometry != GEOM_CHANNEL;
  const bool pery = sI.geometry == GEOM_PERIODIC;
  const bool channel = sI.geometry == GEOM_CHANNEL;
  const bool multiphase = sI.multiphase != 0;

  const Real* __restrict__ Fin = static_cast<const Real*>(sI.f[step & 1]);
  const Real* __restrict__ Gin = static_cast<const Real*>(sI.g[step & 1]);
  Real* __restrict__ Fout = static_cast<Real*>(sI.f[(step + 1) & 1]);
  Real* __restrict__ Gout = static_cast<Real*>(sI.g[(step + 1) & 1]);

  // constants in the compute precision
  const Real omega_f = Real(sI.omega_f), omega_g = Real(sI.omega_g);
  const Real pa = Real(sI.a), pb = Real(sI.b), pR = Real(sI.R), kappa = Real(sI.kappa);
  const Real sqrtTc = Real(sI.sqrtTc), inv_sqrtTc = Real(sI.inv_sqrtTc);
  const Real psi_scale = Real(sI.psi_scale), beta = Real(sI.beta);
  const Real G2 = Real(sI.G2), Gh = Real(sI.Ghalf), Gwet_psiw = Real(sI.Gwet_psiw);
  const Real g_a = Real(sI.g_a), inv_cv = Real(sI.inv_cv);
  const Real T0 = Real(sI.T0), rho_ref = Real(sI.rho_ref), T_ref = Real(sI.T_ref);
  const Real alpha0 = Real(sI.alpha0), u_in = Real(sI.u_in), rho_out = Real(sI.rho_out);
  const Real drho_out = Real(sI.rho_out - sI.rho_ref);
  const Real dT_in = Real(sI.T_in - sI.T_ref), dT_heat = Real(sI.T_heat - sI.T_ref);
  const Real rho_avg_prev = Real(st->rho_avg[(step - 1) & 1]);
  // heater state of the boundary condition that produced the pulled populations (step n-1)
  const bool heat_bc = THERMAL && sI.heater_len > 0 && (step - 1) >= sI.heat_on_step;
  const int hx0 = sI.heater_x0, hx1 = sI.heater_x0 + sI.heater_len;

  // column owned by this thread
  int s, xc;
  if (tid < W) {
    s = tid + 2;
    xc = tile.x0 + tid;
  } else if (tid < W + 4) {
    const int h = tid - W;
    s = (h < 2) ? h : W + h;
    xc = tile.x0 - 2 + s;
  } else {
    s = -1;
    xc = 0;
  }
  int xn = xc;
  bool col_ok = s >= 0;
  if (perx) {
    xn = wrap_index(xc, nx);
  } else {
    col_ok = col_ok && xc >= 0 && xc < nx;
  }
  const bool out_col = tid < W && xc < nx;
  const bool f_col = col_ok && s >= 1 && s <= W + 2;
  // shared-memory neighbours; at the open ends the ghost column repeats the end column
  const int sm = (!perx && xc == 0) ? s : s - 1;
  const int sp = (!perx && xc == nx - 1) ? s : s + 1;
  int xm = xn - 1, xp = xn + 1;
  if (perx) {
    if (xm < 0) xm += nx;
    if (xp >= nx) xp -= nx;
  }
  const bool inl = channel && xn == 0;
  const bool outl = channel && xn == nx - 1;

  // per-thread diagnostics accumulators
  double acc[NPART] = {0.0, 0.0, 0.0, 0.0, 0.0};

  // registers carried between iterations: row r-1 (f collision) and r-2 (g collision)
  Real fp[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) fp[i] = Real(0);
  Real rho_p = Real(1), drho_p = Real(0), ux_p = Real(0), uy_p = Real(0), T_p = T0, dT_p = Real(0),
       coef_p = Real(0);
  Real T_p2 = T0, dT_p2 = Real(0), coef_p2 = Real(0);

  const int nrow = tile.y1 - tile.y0;
  const int kbeg = (MODE == MODE_STEP) ? 0 : (MODE == MODE_FIELDS ? 1 : 2);
  const int kend = (MODE == MODE_STEP) ? nrow + 4 : (MODE == MODE_FIELDS ? nrow + 3 : nrow + 2);
  int k3 = kbeg % 3;

  for (int k = kbeg; k < kend; ++k) {
    const int r = tile.y0 - 2 + k;
    // ===================== Phase A: pull row r, moments, EOS =====================
    const bool row_ok = pery || (r >= 0 && r < ny);
    const int rn = pery ? wrap_index(r, ny) : r;
    Real fc[9], gc[9];
    Real rho_c = Real(1), drho_c = Real(0), ux_c = Real(0), uy_c = Real(0), T_c = T0, dT_c = Real(0),
         coef_c = Real(0);
    if (col_ok && row_ok) {
      const long long node = (long long)rn * pitch + xn;
      if (local) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          fc[i] = ld_ro(Fin + i * plane + node);
          gc[i] = THERMAL ? ld_ro(Gin + i * plane + node) : Real(0);
        }
      } else {
        int rm = rn - 1, rp = rn + 1;
        if (pery) {
          if (rm < 0) rm += ny;
          if (rp >= ny) rp -= ny;
        }
        const bool wlo = !pery && rn == 0;       // links with c_y = +1 come from the bottom wall
        const bool whi = !pery && rn == ny - 1;  // links with c_y = -1 come from the top wall
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          const int cxi = lat_cx(i), cyi = lat_cy(i);
          const bool wall = (cyi == 1 && wlo) || (cyi == -1 && whi);
          const bool unknown = (cxi == 1 && inl) || (cxi == -1 && outl);
          if (wall) {
            // halfway bounce-back (f), anti-bounce-back at the wall temperature (g), Sec. 2.C
            fc[i] = ld_ro(Fin + lat_opp(i) * plane + node);
            if (THERMAL) {
              Real dTw = dT_in;
              if (cyi == 1 && heat_bc) {
                int sx = xn - cxi;
                if (perx) sx = wrap_index(sx, nx);
                if (sx >= hx0 && sx < hx1) dTw = dT_heat;
              }
              gc[i] = -ld_ro(Gin + lat_opp(i) * plane + node) + Real(2) * lat_w<Real>(i) * dTw;
            } else {
              gc[i] = Real(0);
            }
          } else if (!unknown) {
            const int sxx = cxi == 1 ? xm : (cxi == -1 ? xp : xn);
            const int syy = cyi == 1 ? rm : (cyi == -1 ? rp : rn);
            const long long src = (long long)syy * pitch + sxx;
            fc[i] = ld_ro(Fin + i * plane + src);
            gc[i] = THERMAL ? ld_ro(Gin + i * plane + src) : Real(0);
          } else {
            fc[i] = Real(0);
            gc[i] = Real(0);
          }
        }
        if (inl) {
          // velocity inlet (Zou-He non-equilibrium bounce-back), u = (u_in, 0)
          const Real S = fc[0] + fc[2] + fc[4] + Real(2) * (fc[3] + fc[6] + fc[7]);
          const Real rho_b = (S + rho_ref) / (Real(1) - u_in);
          const Real ru = rho_b * u_in;
          if (wlo) {
            fc[8] = fc[2] + fc[5] + fc[6] - fc[4] - fc[7];
            fc[1] = ru - fc[5] - fc[8] + fc[3] + fc[6] + fc[7];
          } else if (whi) {
            fc[5] = fc[4] + fc[7] + fc[8] - fc[2] - fc[6];
            fc[1] = ru - fc[5] - fc[8] + fc[3] + fc[6] + fc[7];
          } else {
            const Real h = Real(0.5) * (fc[2] - fc[4]);
            fc[1] = fc[3] + Real(2.0 / 3.0) * ru;
            fc[5] = fc[7] - h + ru * Real(1.0 / 6.0);
            fc[8] = fc[6] + h + ru * Real(1.0 / 6.0);
          }
          if (THERMAL) {
            // anti-bounce-back at the inlet temperature
            if (!wlo) gc[5] = -ld_ro(Gin + 7 * plane + node) + Real(2) * lat_w<Real>(5) * dT_in;
            if (!whi) gc[8] = -ld_ro(Gin + 6 * plane + node) + Real(2) * lat_w<Real>(8) * dT_in;
            gc[1] = -ld_ro(Gin + 3 * plane + node) + Real(2) * lat_w<Real>(1) * dT_in;
          }
        }
        if (outl) {
          // pressure outlet (Zou-He), rho = rho_out, u_y = 0
          if (wlo) {
            fc[7] = fc[2] + fc[5] + fc[6] - fc[4] - fc[8];
            fc[3] = drho_out - (fc[0] + fc[1] + fc[2] + fc[4] + fc[5] + fc[6] + fc[7] + fc[8]);
          } else if (whi) {
            fc[6] = fc[4] + fc[7] + fc[8] - fc[2] - fc[5];
            fc[3] = drho_out - (fc[0] + fc[1] + fc[2] + fc[4] + fc[5] + fc[6] + fc[7] + fc[8]);
          } else {
            const Real S = fc[0] + fc[2] + fc[4] + Real(2) * (fc[1] + fc[5] + fc[8]);
            const Real ru = S + rho_ref - rho_out;  // rho_out * u_x
            const Real h = Real(0.5) * (fc[2] - fc[4]);
            fc[3] = fc[1] - Real(2.0 / 3.0) * ru;
            fc[7] = fc[5] + h - ru * Real(1.0 / 6.0);
            fc[6] = fc[8] - h - ru * Real(1.0 / 6.0);
          }
          if (THERMAL) {
            // zero temperature gradient: the post-stream populations of node nx-2
            const long long col = xn;
            gc[3] = ld_ro(Gin + 3 * plane + (long long)rn * pitch + col);
            if (!wlo) gc[6] = ld_ro(Gin + 6 * plane + (long long)(rn - 1) * pitch + col);
            if (!whi) gc[7] = ld_ro(Gin + 7 * plane + (long long)(rn + 1) * pitch + col);
          }
        }
      }

      // moments, Eqs. 4, 6, 17 (deviation sums; the rest-state parts carry no momentum)
      drho_c = ((fc[0] + fc[1]) + (fc[2] + fc[3])) + ((fc[4] + fc[5]) + (fc[6] + fc[7])) + fc[8];
      rho_c = rho_ref + drho_c;
      const Real jx = (fc[1] - fc[3]) + (fc[5] - fc[6]) + (fc[8] - fc[7]);
      const Real jy = (fc[2] - fc[4]) + (fc[5] + fc[6]) - (fc[7] + fc[8]);
      const Real inv_rho = Real(1) / rho_c;
      ux_c = jx * inv_rho;
      uy_c = jy * inv_rho;
      if (THERMAL) {
        dT_c = ((gc[0] + gc[1]) + (gc[2] + gc[3])) + ((gc[4] + gc[5]) + (gc[6] + gc[7])) + gc[8];
        T_c = T_ref + dT_c;
      }

      // Peng-Robinson EOS (Eq. 12), pseudopotential (Eq. 11), (dp/dT)_rho
      Real psi = Real(0), p = rho_c * Real(1.0 / 3.0), dpdT = Real(0);
      bool bad = !(rho_c > Real(0));
      if (multiphase) {
        const Real br = pb * rho_c;
        const Real inv1 = Real(1) / (Real(1) - br);
        const Real rr_den = rho_c * rho_c / (Real(1) + br * (Real(2) - br));
        Real alpha, sa = Real(0), sT = Real(0);
        if (THERMAL) {
          sT = sqrt(T_c);
          sa = Real(1) + kappa * (Real(1) - sT * inv_sqrtTc);
          alpha = sa * sa;
        } else {
          alpha = alpha0;
        }
        p = rho_c * pR * T_c * inv1 - pa * alpha * rr_den;
        const Real rad = (p - rho_c * Real(1.0 / 3.0)) * psi_scale;
        bad = bad || !(br < Real(1)) || !(rad >= Real(0));
        psi = sqrt(fmax(rad, Real(0)));
        if (THERMAL) {
          const Real dalpha = -kappa * sa / (sT * sqrtTc);
          dpdT = rho_c * pR * inv1 - pa * dalpha * rr_den;
        }
      }
      if (THERMAL) {
        bad = bad || !isfinite(T_c);
        coef_c = T_c * (Real(1) - dpdT * inv_rho * inv_cv);
      }
      if (bad) atomicOr(&st->status, STATUS_UNSTABLE);
      sPsi[k3][s] = psi;
      if (THERMAL && MODE == MODE_STEP && tid < W) {
#pragma unroll
        for (int i = 0; i < 9; ++i) sG[k3][i][tid] = gc[i];
      }
      const bool out_row = r >= tile.y0 && r < tile.y1;
      if ((MODE == MODE_STEP || MODE == MODE_MOMENTS) && out_col && out_row) {
        acc[0] += (double)rho_c;
        acc[1] += (double)T_c;
        if (THERMAL && !pery && rn == 0 && xn >= hx0 && xn < hx1) acc[2] += (double)T_c;
        if (MODE == MODE_STEP && channel && rn == ny / 2 && (xn == 1 || xn == nx - 2)) {
          if (xn == 1) st->p_probe[0] = (double)p;
          if (xn == nx - 2) st->p_probe[1] = (double)p;
          __threadfence();
        }
      }
      if (MODE == MODE_POPS && out_col && out_row) {
        const long long o = (long long)rn * pitch + xn;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          Fout[i * plane + o] = fc[i];
          if (THERMAL) Gout[i * plane + o] = gc[i];
        }
      }
    }
    if (MODE == MODE_POPS || MODE == MODE_MOMENTS) {
      k3 = (k3 == 2) ? 0 : k3 + 1;
      continue;
    }
    __syncthreads();

    // ============ Phase B: row q = r - 1: force, u_act, f collision ============
    const int q = r - 1;
    const int k3m1 = (k3 == 0) ? 2 : k3 - 1;  // slot of row r-1
    const int k3m2 = (k3m1 == 0) ? 2 : k3m1 - 1;  // slot of row r-2
    // STEP needs u_act from row y0 - 1 (divergence at y0); FIELDS only on its output rows
    const int qmin = (MODE == MODE_STEP) ? tile.y0 - 1 : tile.y0;
    if (q >= qmin) {
      const bool qrow_ok = pery || (q >= 0 && q < ny);
      if (f_col && qrow_ok) {
        const bool sol_m = !pery && q == 0;       // row q-1 is the bottom wall
        const bool sol_p = !pery && q == ny - 1;  // row q+1 is the top wall
        Real Fx = Real(0), Fy = Real(0);
        if (multiphase) {
          const Real pc = sPsi[k3m1][s];
          const Real pE = sPsi[k3m1][sp], pW = sPsi[k3m1][sm];
          Real pN = Real(0), pNE = Real(0), pNW = Real(0), pS = Real(0), pSE = Real(0), pSW = Real(0);
          if (!sol_p) {
            pN = sPsi[k3][s];
            pNE = sPsi[k3][sp];
            pNW = sPsi[k3][sm];
          }
          if (!sol_m) {
            pS = sPsi[k3m2][s];
            pSE = sPsi[k3m2][sp];
            pSW = sPsi[k3m2][sm];
          }
          // Eq. 9 sums over fluid neighbours: sum G_i psi(x1) c_i and sum G_i psi(x1)^2 c_i
          const Real s1x = G2 * (pE - pW) + Gh * ((pNE - pNW) + (pSE - pSW));
          const Real s1y = G2 * (pN - pS) + Gh * ((pNE + pNW) - (pSE + pSW));
          const Real s2x = G2 * (pE * pE - pW * pW) + Gh * ((pNE * pNE - pNW * pNW) + (pSE * pSE - pSW * pSW));
          const Real s2y = G2 * (pN * pN - pS * pS) + Gh * ((pNE * pNE + pNW * pNW) - (pSE * pSE + pSW * pSW));
          const Real mix = Real(0.5) * (Real(1) - beta);
          Fx = -beta * pc * s1x - mix * s2x;
          Fy = -beta * pc * s1y - mix * s2y;
          // Eq. 15: solid neighbours, sum_i w_i c_iy = -1/6 below, +1/6 above
          Real wy = Real(0);
          if (sol_m) wy -= Real(1.0 / 6.0);
          if (sol_p) wy += Real(1.0 / 6.0);
          Fy -= Gwet_psiw * pc * wy;
        }
        Fy -= (rho_p - rho_avg_prev) * g_a;  // Eq. 14, gravity along -y
        const Real inv_rho = Real(1) / rho_p;
        const Real dux = Fx * inv_rho, duy = Fy * inv_rho;
        const Real uax = ux_p + Real(0.5) * dux, uay = uy_p + Real(0.5) * duy;  // Eq. 7
        sUx[k3m1][s] = uax;
        sUy[k3m1][s] = uay;
        const bool out_q = out_col && q >= tile.y0 && q < tile.y1;
        if (MODE == MODE_STEP && out_q) {
          // BGK toward f^eq(rho, u_eq) (Eqs. 2-3) plus the exact-difference term (Eq. 5),
          // written as the difference of the two equilibria expanded in du
          const Real sx = Real(2) * ux_p + dux, sy = Real(2) * uy_p + duy;
          const Real usq = ux_p * ux_p + uy_p * uy_p;
          const Real dsum = dux * sx + duy * sy;
          const long long o = (long long)q * pitch + xn;
#pragma unroll
          for (int i = 0; i < 9; ++i) {
            const Real cu = Real(lat_cx(i)) * ux_p + Real(lat_cy(i)) * uy_p;
            const Real cd = Real(lat_cx(i)) * dux + Real(lat_cy(i)) * duy;
            const Real cs = Real(lat_cx(i)) * sx + Real(lat_cy(i)) * sy;
            const Real wi = lat_w<Real>(i);
            const Real feq = wi * (drho_p + rho_p * (Real(3) * cu + Real(4.5) * cu * cu - Real(1.5) * usq));
            const Real Fi = wi * rho_p * (Real(3) * cd + Real(4.5) * cd * cs - Real(1.5) * dsum);
            Fout[i * plane + o] = fp[i] + omega_f * (feq - fp[i]) + Fi;
          }
          if (channel && xn == 0) acc[3] += (double)rho_p * (double)uax;
          if (channel && xn == nx - 1) acc[4] += (double)rho_p * (double)uax;
        }
        if (MODE == MODE_FIELDS && out_q) {
          double* out = static_cast<double*>(sI.f[(step + 1) & 1]);
          const long long n = (long long)nx * ny;
          const long long o = (long long)q * nx + xn;
          out[o] = (double)rho_p;
          out[n + o] = (double)uax;
          out[2 * n + o] = (double)uay;
          out[3 * n + o] = (double)T_p;
        }
      }
    }
    __syncthreads();

    // ============ Phase C: row q2 = r - 2: source and g collision ============
    if (THERMAL && MODE == MODE_STEP) {
      const int q2 = r - 2;
      if (out_col && q2 >= tile.y0 && q2 < tile.y1) {
        // second-order central differences of u_act; zero at solid rows, ghost copy at open ends
        const Real uxE = sUx[k3m2][sp], uxW = sUx[k3m2][sm];
        const Real uyN = (!pery && q2 == ny - 1) ? Real(0) : sUy[k3m1][s];
        const int k3m3 = (k3m2 == 0) ? 2 : k3m2 - 1;
        const Real uyS = (!pery && q2 == 0) ? Real(0) : sUy[k3m3][s];
        const Real divu = Real(0.5) * (uxE - uxW) + Real(0.5) * (uyN - uyS);
        const Real phi = coef_p2 * divu;  // second Eq. 19
        const Real uax = sUx[k3m2][s], uay = sUy[k3m2][s];
        const Real usq = uax * uax + uay * uay;
        const long long o = (long long)q2 * pitch + xn;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          const Real cu = Real(lat_cx(i)) * uax + Real(lat_cy(i)) * uay;
          const Real wi = lat_w<Real>(i);
          const Real geq = wi * (dT_p2 + T_p2 * (Real(3) * cu + Real(4.5) * cu * cu - Real(1.5) * usq));
          const Real gi = sG[k3m2][i][tid];
          Gout[i * plane + o] = gi + omega_g * (geq - gi) + wi * phi;  // Eq. 16
        }
      }
    }

    // rotate the carried rows
    T_p2 = T_p;
    dT_p2 = dT_p;
    coef_p2 = coef_p;
#pragma unroll
    for (int i = 0; i < 9; ++i) fp[i] = fc[i];
    rho_p = rho_c;
    drho_p = drho_c;
    ux_p = ux_c;
    uy_p = uy_c;
    T_p = T_c;
    dT_p = dT_c;
    coef_p = coef_c;
    k3 = (k3 == 2) ? 0 : k3 + 1;
  }

  if (MODE != MODE_STEP && MODE != MODE_MOMENTS) return;

  // ---------------- per-tile partials and the last-CTA fold ----------------
  block_sum<BLOCK>(acc, sRed);
  if (tid == 0) {
    double* part = sI.partials + (long long)tile.local * NPART;
#pragma unroll
    for (int j = 0; j < NPART; ++j) part[j] = acc[j];
    __threadfence();
    const unsigned ticket = atomicAdd(&st->counter, 1u);
    sLast = (ticket == (unsigned)(tile.ntiles - 1));
  }
  __syncthreads();
  if (!sLast) return;
  __threadfence();
  double tot[NPART] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int t = tid; t < tile.ntiles; t += BLOCK) {
#pragma unroll
    for (int j = 0; j < NPART; ++j) tot[j] += __ldcg(sI.partials + (long long)t * NPART + j);
  }
  __syncthreads();
  block_sum<BLOCK>(tot, sRed);
  if (tid == 0) {
    const double n = (double)nx * (double)ny;
    const double mass = tot[0], energy = tot[1];
    if (MODE == MODE_STEP) {
      double dtstar = 0.0;
      const bool heat_now = THERMAL && sI.heater_len > 0 && step >= sI.heat_on_step && !pery;
      if (heat_now) {
        int lo = hx0 < 0 ? 0 : hx0, hi = hx1 > nx ? nx : hx1;
        if (hi > lo) {
          const double tnb = tot[2] / (double)(hi - lo);
          dtstar = (sI.T_heat - tnb) / (sI.T_heat - energy / n);
        }
      }
      double* rec = sI.ring + (step % RING) * NDIAG;
      rec[0] = (double)step;
      rec[1] = mass;
      rec[2] = energy;
      rec[3] = mass / n;
      rec[4] = channel ? __ldcg(&st->p_probe[0]) - __ldcg(&st->p_probe[1]) : 0.0;
      rec[5] = dtstar;
      rec[6] = channel ? tot[3] : 0.0;
      rec[7] = channel ? tot[4] : 0.0;
      st->rho_avg[step & 1] = mass / n;
      st->step = step + 1;
      st->local_read = 0;
    } else {
      st->rho_avg[(step - 1) & 1] = mass / n;
    }
    st->counter = 0u;
  }
}

// ---------------------------------------------------------------------------
// Initialisation: f = f^eq(rho, u) (Eq. 3), g = g^eq(T, u) (Eq. 18) into buffer 0,
// stored in the library's storage form (deviations in FP32).
// ---------------------------------------------------------------------------
template <typename Real>
__device__ __forceinline__ void write_equilibrium(const Inst& I, long long node, double rho, double ux,
                                                  double uy, double T) {
  Real* F = static_cast<Real*>(I.f[0]);
  Real* Gb = static_cast<Real*>(I.g[0]);
  const double usq = ux * ux + uy * uy;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const double cu = lat_cx(i) * ux + lat_cy(i) * uy;
    const double w = lat_w<double>(i);
    const double poly = 3.0 * cu + 4.5 * cu * cu - 1.5 * usq;
    F[i * I.plane + node] = Real(w * ((rho - I.rho_ref) + rho * poly));
    Gb[i * I.plane + node] = Real(w * ((T - I.T_ref) + T * poly));
  }
}

template <typename Real>
__global__ void lbm_init_fields_kernel(const Inst* __restrict__ insts, const double* __restrict__ fields, int has_T) {
  const Inst I = insts[0];
  const long long n = (long long)I.nx * I.ny;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(k / I.nx), x = (int)(k - (long long)y * I.nx);
    const double T = has_T ? fields[3 * n + k] : I.T0;
    write_equilibrium<Real>(I, (long long)y * I.pitch + x, fields[k], fields[n + k], fields[2 * n + k], T);
  }
}

// splitmix64 (Steele, Lea & Flood, OOPSLA 2014) as a counter-based hash.
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename Real>
__global__ void lbm_init_builtin_kernel(const Inst* __restrict__ insts, InitSpec spec) {
  const Inst I = insts[0];
  const long long n = (long long)I.nx * I.ny;
  const double cx = 0.5 * (I.nx - 1), cy = 0.5 * (I.ny - 1);
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const int y = (int)(k / I.nx), x = (int)(k - (long long)y * I.nx);
    double rho = spec.rho_out;
    if (spec.kind == 1) {
      const double r = sqrt((x - cx) * (x - cx) + (y - cy) * (y - cy));
      rho = 0.5 * (spec.rho_in + spec.rho_out) - 0.5 * (spec.rho_in - spec.rho_out) * tanh(2.0 * (r - spec.radius) / spec.width);
      if (spec.amp != 0.0) {
        const unsigned long long key =
            spec.seed ^ ((unsigned long long)spec.instance << 40) ^ (unsigned long long)k;
        const double u = (double)(splitmix64(key) >> 11) * (1.0 / 9007199254740992.0);
        rho *= 1.0 + spec.amp * (2.0 * u - 1.0);
      }
    }
    write_equilibrium<Real>(I, (long long)y * I.pitch + x, rho, 0.0, 0.0, spec.T0);
  }
}

// ---------------------------------------------------------------------------
// Host launchers for one storage precision.
// ---------------------------------------------------------------------------
template <typename Real, bool THERMAL, int W>
cudaError_t launch_cols(int mode, const Inst* d_inst, const Tile* d_tiles, int ntiles, cudaStream_t s) {
  dim3 grid(ntiles), block(W + 32);
  switch (mode) {
    case MODE_STEP: lbm_fused_kernel<Real, THERMAL, W, MODE_STEP><<<grid, block, 0, s>>>(d_inst, d_tiles); break;
    case MODE_FIELDS: lbm_fused_kernel<Real, THERMAL, W, MODE_FIELDS><<<grid, block, 0, s>>>(d_inst, d_tiles); break;
    case MODE_POPS: lbm_fused_kernel<Real, THERMAL, W, MODE_POPS><<<grid, block, 0, s>>>(d_inst, d_tiles); break;
    case MODE_MOMENTS: lbm_fused_kernel<Real, THERMAL, W, MODE_MOMENTS><<<grid, block, 0, s>>>(d_inst, d_tiles); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_precision(int thermal, int cols, int mode, const Inst* d_inst, const Tile* d_tiles, int ntiles,
                             cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  if (thermal) {
    switch (cols) {
      case 64: return launch_cols<Real, true, 64>(mode, d_inst, d_tiles, ntiles, s);
      case 128: return launch_cols<Real, true, 128>(mode, d_inst, d_tiles, ntiles, s);
      case 256:
        // three rows of nine FP64 planes for 256 columns exceed the 48 KB static shared memory
        if (sizeof(Real) == 8) return cudaErrorInvalidValue;
        return launch_cols<Real, true, (sizeof(Real) == 8 ? 128 : 256)>(mode, d_inst, d_tiles, ntiles, s);
    }
  } else {
    switch (cols) {
      case 64: return launch_cols<Real, false, 64>(mode, d_inst, d_tiles, ntiles, s);
      case 128: return launch_cols<Real, false, 128>(mode, d_inst, d_tiles, ntiles, s);
      case 256: return launch_cols<Real, false, 256>(mode, d_inst, d_tiles, ntiles, s);
    }
  }
  return cudaErrorInvalidValue;
}

template <typename Real>
cudaError_t launch_init_fields_t(const Inst* d_inst, int nx, int ny, const double* d_fields, int has_T,
                                 cudaStream_t s) {
  const long long n = (long long)nx * ny;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  lbm_init_fields_kernel<Real><<<blocks, 256, 0, s>>>(d_inst, d_fields, has_T);
  return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_init_builtin_t(const Inst* d_inst, int nx, int ny, InitSpec spec, cudaStream_t s) {
  const long long n = (long long)nx * ny;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  lbm_init_builtin_kernel<Real><<<blocks, 256, 0, s>>>(d_inst, spec);
  return cudaGetLastError();
}

}  // namespace pplbm
