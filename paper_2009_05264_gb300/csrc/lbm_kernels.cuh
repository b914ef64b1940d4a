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
// Work decomposition: a CTA of B threads (64, 128 or 256) owns B - 8 output
// columns [x0, x0 + B - 8) and a band of rows [y0, y1), and marches up the band
// one row per iteration.  Its threads map to the columns [x0 - 2, x0 + B - 6): the
// outputs plus two halo columns per side (the last 4 lanes idle, so every CTA's
// output starts on a 32-byte sector).  The force at a node needs psi on its 8
// neighbours and the divergence of u_act in the g source needs u_act (hence the
// force) on the 4 neighbours, so psi is needed two nodes out: the CTA keeps
// three-row rings of psi and u_act in shared memory.  At iteration k it pulls
// row r = y0 - 2 + k (phase A: boundary fill, moments, EOS), computes force, u_act
// and the f collision of row r - 1 (phase B) and the g collision of row r - 2
// (phase C), with a barrier after A and after B.  Each thread's pulled
// populations are staged in its own shared-memory ring by cp.async, one row ahead,
// so the loads of the next row are in flight during the arithmetic of this one.
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
// D2Q9 weights.  In FP32 the rounded 4/9, 1/9, 1/36 sum to 1 + 7.6e-9, which would
// create mass (and energy) in every collision in proportion to the stored deviation;
// the FP32 set below (1/36 lowered by one ulp) sums to exactly 1.
template <typename Real>
struct LatWeights {
  __host__ __device__ static constexpr Real w0() { return Real(4.0 / 9.0); }
  __host__ __device__ static constexpr Real w1() { return Real(1.0 / 9.0); }
  __host__ __device__ static constexpr Real w5() { return Real(1.0 / 36.0); }
};
template <>
struct LatWeights<float> {
  __host__ __device__ static constexpr float w0() { return 0x1.c71c72p-2f; }
  __host__ __device__ static constexpr float w1() { return 0x1.c71c72p-4f; }
  __host__ __device__ static constexpr float w5() { return 0x1.c71c70p-6f; }
};
template <typename Real>
__host__ __device__ constexpr Real lat_w(int i) {
  return i == 0 ? LatWeights<Real>::w0() : (i <= 4 ? LatWeights<Real>::w1() : LatWeights<Real>::w5());
}

__device__ __forceinline__ int wrap_index(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

__device__ __forceinline__ float ld_ro(const float* p) { return __ldg(p); }
__device__ __forceinline__ double ld_ro(const double* p) { return __ldg(p); }

// Bounds-checked build (compiled with -DLBM_BOUNDS_CHECK, for tests): before each global access
// of the step and initialisation kernels, idx_ok checks the element index k against the n
// elements of the buffer it addresses.  An index outside [0, n) sets STATUS_BOUNDS in the
// instance's status word and counts the access in bounds_hits, and the caller skips the
// access (a load reads 0, a store goes to a scratch word), so nothing faults or traps.  In the
// default build idx_ok is the constant true and every check compiles away.
#ifdef LBM_BOUNDS_CHECK
__device__ inline bool idx_ok(InstState* st, long long k, long long n) {
  if (k >= 0 && k < n) return true;
  atomicOr(&st->status, STATUS_BOUNDS);
  atomicAdd(&st->bounds_hits, 1u);
  return false;
}
template <typename Real>
__device__ inline Real& bounds_sink() {
  __shared__ Real sink;  // where a rejected store goes
  return sink;
}
#else
__device__ __forceinline__ constexpr bool idx_ok(InstState*, long long, long long) { return true; }
#endif

// Reciprocal and reciprocal square root.  FP32: MUFU approximations (about 2 ulp).  FP64: the
// PTX approximations rcp.approx / rsqrt.approx (about 23 correct bits) refined by two
// Newton-Raphson steps on f(y) = 1/y - x and f(y) = 1/y^2 - x (each step squares the relative
// error), which ends within a few ulp of the correctly rounded result in fewer FP64
// instructions than an IEEE division or square root on this GPU's narrow FP64 pipe; inputs are
// positive normal numbers here (densities, temperatures, psi radicands).
__device__ __forceinline__ float fast_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double fast_rcp(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;\n" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);  // relative error of y
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}
__device__ __forceinline__ float fast_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double fast_rsqrt(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;\n" : "=d"(y) : "d"(x));
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double e = fma(-x, y * y, 1.0);  // 1 - x y^2
    y = fma(0.5 * y, e, y);
  }
  return y;
}
__device__ __forceinline__ float fast_sqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
__device__ __forceinline__ double fast_sqrt(double x) { return x > 0.0 ? x * fast_rsqrt(x) : 0.0; }

// Asynchronous global -> shared copies of one element (cp.async, Ampere and later).
__device__ __forceinline__ void cp_async_elem(float* smem, const float* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_elem(double* smem, const double* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
// Wait until at most N of this thread's most recent copy groups are still in flight.
template <int N>
__device__ __forceinline__ void cp_async_wait_lookahead() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Ring depths of the staged populations: f of rows r+1 (in flight), r (pulled
// now) and r-1 (collided now); g additionally keeps row r-2 (collided now).
constexpr int F_SLOTS = 3;
constexpr int G_SLOTS = 4;

// A CTA of B threads owns B - 8 output columns: its threads map to the columns
// [x0 - 2, x0 + B - 6), i.e. the output columns plus two halo columns per side, and
// the last 4 lanes idle, so that every CTA's output starts on a 32-byte sector.
template <int B>
__host__ __device__ constexpr int out_cols() { return B - 8; }

template <typename Real, bool THERMAL, int B>
constexpr size_t fused_smem_bytes() {
  return sizeof(Real) * (size_t)(B - 4) * (9 * F_SLOTS + (THERMAL ? 9 * G_SLOTS : 0) + 9);
}

// Rows the interior path stages ahead of the row it computes (its rings hold f of rows
// r + LOOKAHEAD .. r - 1 and g of rows r + LOOKAHEAD .. r - 2).  One row: the copies of row r + 1
// are in flight during the arithmetic of row r (deeper staging measured slower on GB300: the
// larger rings leave less room for L1).
constexpr int LOOKAHEAD = 1;
constexpr int FI_SLOTS = 2 + LOOKAHEAD;
constexpr int GI_SLOTS = 3 + LOOKAHEAD;
template <typename Real, bool THERMAL, int B>
constexpr size_t interior_smem_bytes() {
  return sizeof(Real) * (size_t)(B - 4) * (9 * FI_SLOTS + (THERMAL ? 9 * GI_SLOTS : 0) + 9);
}
// Dynamic shared memory of a step-kernel instantiation (the interior path's layout is larger).
template <typename Real, bool THERMAL, int B, bool INTERIOR>
constexpr size_t step_smem_bytes() {
  return INTERIOR && interior_smem_bytes<Real, THERMAL, B>() > fused_smem_bytes<Real, THERMAL, B>()
             ? interior_smem_bytes<Real, THERMAL, B>()
             : fused_smem_bytes<Real, THERMAL, B>();
}

// ---------------------------------------------------------------------------
// Per-instance constants of the update, converted once per CTA to the compute
// precision (the instance descriptor holds them in FP64).
// ---------------------------------------------------------------------------
template <typename Real>
struct KConst {
  Real omega_f, omega_g, a, b, R, kappa, inv_sqrtTc, psi_scale, beta, G2, Gh, mix, g_a, inv_cv;
  Real T0, rho_ref, T_ref, alpha0, u_in, drho_out, dT_in, dT_heat;
  // FP32 pseudopotential reference state (zero in FP64)
  Real inv_u1r, inv_Dr, sqrtT_r, sa_r, rr2_Dr, rad_ref, psi_ref, p_ref;
  // force on a row next to the bottom wall: wall0 + d * wall1 (the top wall: minus that)
  Real wall0, wall1;
  Real rho_ref_minus_avg;  // rho_ref - rho_avg of the previous step (buoyancy, Eq. 14)
  Real drho_vapor;         // rho_vapor - rho_ref: vapour when drho < drho_vapor
  // products of the constants above, formed once (host doubles): R / (1 - b rho_ref),
  // a / D(rho_ref), 2 b rho_ref, -kappa / sqrt(Tc), a rho_ref^2 / D(rho_ref)
  Real R_u1r, a_Dr, twob_rr, nk_sTc, a_rr2_Dr;
};

// Every member is a conversion of a descriptor value (derived values are formed once, on the
// host, in fill_inst), so the host's copy (kernel parameter) and a CTA's copy (shared memory)
// are bit-identical.
template <typename Real>
__host__ __device__ inline void fill_consts(KConst<Real>& c, const Inst& I, double rho_avg_prev) {
  c.omega_f = Real(I.omega_f);
  c.omega_g = Real(I.omega_g);
  c.a = Real(I.a);
  c.b = Real(I.b);
  c.R = Real(I.R);
  c.kappa = Real(I.kappa);
  c.inv_sqrtTc = Real(I.inv_sqrtTc);
  c.psi_scale = Real(I.psi_scale);
  c.beta = Real(I.beta);
  c.G2 = Real(I.G2);
  c.Gh = Real(I.Ghalf);
  c.mix = Real(I.mix);
  c.g_a = Real(I.g_a);
  c.inv_cv = Real(I.inv_cv);
  c.T0 = Real(I.T0);
  c.rho_ref = Real(I.rho_ref);
  c.T_ref = Real(I.T_ref);
  c.alpha0 = Real(I.alpha0);
  c.u_in = Real(I.u_in);
  c.drho_out = Real(I.drho_out);
  c.dT_in = Real(I.dT_in);
  c.dT_heat = Real(I.dT_heat);
  c.inv_u1r = Real(I.inv_u1r);
  c.inv_Dr = Real(I.inv_Dr);
  c.sqrtT_r = Real(I.sqrtT_r);
  c.sa_r = Real(I.sa_r);
  c.rr2_Dr = Real(I.rr2_Dr);
  c.rad_ref = Real(I.rad_ref);
  c.psi_ref = Real(I.psi_ref);
  c.p_ref = Real(I.p_ref);
  c.wall0 = Real(I.wall0);
  c.wall1 = Real(I.wall1);
  c.rho_ref_minus_avg = Real(I.rho_ref - rho_avg_prev);
  c.drho_vapor = Real(I.drho_vapor);
  c.R_u1r = Real(I.R_u1r);
  c.a_Dr = Real(I.a_Dr);
  c.twob_rr = Real(I.twob_rr);
  c.nk_sTc = Real(I.nk_sTc);
  c.a_rr2_Dr = Real(I.a_rr2_Dr);
}

// Kernel parameter of a launch over one instance: its descriptor and converted constants.
template <typename Real>
struct KParams {
  Inst I;
  KConst<Real> C;
};

// ---------------------------------------------------------------------------
// Node-level pieces of the step, shared by the kernels below.
// ---------------------------------------------------------------------------

// Where a node sits relative to the boundaries of Sec. 2.C.
struct NodeBC {
  bool wlo, whi;  // links with c_y = +1 / -1 come from the bottom / top wall
  bool inl, outl; // velocity inlet (x = 0) / pressure outlet (x = nx - 1)
  bool top;       // pool top row: links with c_y = -1 come from above the free surface
};

// Complete the pulled populations of a boundary node in place.  Wall links were
// pulled from the node's own opposite population (halfway bounce-back); here g on
// those links gets the anti-bounce-back sign flip and wall temperature, and the
// links from outside an open end are set by the Zou-He conditions.
template <typename Real, bool THERMAL>
__device__ __forceinline__ void boundary_fill(Real (&fc)[9], Real (&gc)[9], const NodeBC& nb, const Inst& I,
                                              const KConst<Real>& C, const Real* __restrict__ Gin, int plane,
                                              int pitch, int node, int xn, bool perx, long long step) {
  const Real rho_ref = C.rho_ref;
  const Real dT_in = C.dT_in;
  // element k of the g buffer (0 outside it, in a bounds-checked build)
  auto gload = [&](int k) { return idx_ok(I.st, k, 9LL * plane) ? ld_ro(Gin + k) : Real(0); };
  if (THERMAL && (nb.wlo || nb.whi)) {
    // anti-bounce-back at the wall temperature (the heater heats the bottom wall
    // once the boundary condition of step heat_on_step has been applied)
    const bool heat_bc = I.heater_len > 0 && (step - 1) >= I.heat_on_step;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int cxi = lat_cx(i), cyi = lat_cy(i);
      if ((cyi == 1 && nb.wlo) || (cyi == -1 && nb.whi)) {
        Real dTw = dT_in;
        if (cyi == 1 && heat_bc) {
          int sx = xn - cxi;
          if (perx) sx = wrap_index(sx, I.nx);
          if (sx >= I.heater_x0 && sx < I.heater_x0 + I.heater_len) dTw = C.dT_heat;
        }
        gc[i] = -gc[i] + Real(2) * lat_w<Real>(i) * dTw;
      }
    }
  }
  if (nb.inl) {
    // velocity inlet (Zou-He non-equilibrium bounce-back), u = (u_in, 0)
    const Real u_in = C.u_in;
    const Real S = fc[0] + fc[2] + fc[4] + Real(2) * (fc[3] + fc[6] + fc[7]);
    const Real rho_b = (S + rho_ref) / (Real(1) - u_in);
    const Real ru = rho_b * u_in;
    if (nb.wlo) {
      fc[8] = fc[2] + fc[5] + fc[6] - fc[4] - fc[7];
      fc[1] = ru - fc[5] - fc[8] + fc[3] + fc[6] + fc[7];
    } else if (nb.whi) {
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
      if (!nb.wlo) gc[5] = -gload(7 * plane + node) + Real(2) * lat_w<Real>(5) * dT_in;
      if (!nb.whi) gc[8] = -gload(6 * plane + node) + Real(2) * lat_w<Real>(8) * dT_in;
      gc[1] = -gload(3 * plane + node) + Real(2) * lat_w<Real>(1) * dT_in;
    }
  }
  if (nb.outl) {
    // pressure outlet (Zou-He), rho = rho_out, u_y = 0
    const Real drho_out = C.drho_out;
    if (nb.wlo) {
      fc[7] = fc[2] + fc[5] + fc[6] - fc[4] - fc[8];
      fc[3] = drho_out - (fc[0] + fc[1] + fc[2] + fc[4] + fc[5] + fc[6] + fc[7] + fc[8]);
    } else if (nb.whi) {
      fc[6] = fc[4] + fc[7] + fc[8] - fc[2] - fc[5];
      fc[3] = drho_out - (fc[0] + fc[1] + fc[2] + fc[4] + fc[5] + fc[6] + fc[7] + fc[8]);
    } else {
      const Real S = fc[0] + fc[2] + fc[4] + Real(2) * (fc[1] + fc[5] + fc[8]);
      const Real ru = S - drho_out;  // rho_out * u_x
      const Real h = Real(0.5) * (fc[2] - fc[4]);
      fc[3] = fc[1] - Real(2.0 / 3.0) * ru;
      fc[7] = fc[5] + h - ru * Real(1.0 / 6.0);
      fc[6] = fc[8] - h - ru * Real(1.0 / 6.0);
    }
    if (THERMAL) {
      // zero temperature gradient: all nine post-stream populations of node nx-2, its
      // wall links (anti-bounce-back at the wall temperature) included
      const int xu = xn - 1;
      const bool heat_bc = I.heater_len > 0 && (step - 1) >= I.heat_on_step;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        const int cxi = lat_cx(i), cyi = lat_cy(i);
        if ((cyi == 1 && nb.wlo) || (cyi == -1 && nb.whi)) {
          const int sx = xu - cxi;
          const Real dTw = (cyi == 1 && heat_bc && sx >= I.heater_x0 && sx < I.heater_x0 + I.heater_len)
                               ? C.dT_heat : dT_in;
          gc[i] = -gload(lat_opp(i) * plane + node - 1) + Real(2) * lat_w<Real>(i) * dTw;
        } else {
          gc[i] = gload(i * plane + node - 1 - cyi * pitch - cxi);
        }
      }
    }
  }
  if (nb.top) {
    // pool top (free surface): Zou-He with rho = rho_out, u_x = 0 for the populations from
    // above (c_y = -1: 4, 7, 8), then zero temperature gradient: every g of the node below
    const Real drho_top = C.drho_out;
    const Real S = fc[0] + fc[1] + fc[3] + Real(2) * (fc[2] + fc[5] + fc[6]);
    const Real ru = S - drho_top;  // rho_out * u_y
    const Real h = Real(0.5) * (fc[1] - fc[3]);
    fc[4] = fc[2] - Real(2.0 / 3.0) * ru;
    fc[7] = fc[5] + h - ru * Real(1.0 / 6.0);
    fc[8] = fc[6] - h - ru * Real(1.0 / 6.0);
    if (THERMAL) {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        int sx = xn - lat_cx(i);
        if (perx) sx = wrap_index(sx, I.nx);
        gc[i] = gload(i * plane + (node - pitch) - xn + sx - lat_cy(i) * pitch);
      }
    }
  }
}

// Macroscopic state of one node (compute precision; deviations from the references).
template <typename Real>
struct NodeState {
  Real rho, drho, ux, uy, T, dT, coef;  // coef = T (1 - (dp/dT)_rho / (rho c_v)) of the source
  Real inv_rho;                          // 1 / rho
  Real hmc;                              // Hazi-Markus form: T (dp/dT)_rho / (rho^2 c_v); coef is then T
  Real dpsi;                             // psi - psi_ref (psi itself in FP64)
  Real p;                                // EOS pressure (diagnostics)
  bool bad;                              // outside the EOS domain
};

// Moments (Eqs. 4, 6, 17), Peng-Robinson EOS (Eq. 12), pseudopotential (Eq. 11) and
// (dp/dT)_rho of one node.  In FP32 psi is evaluated as psi - psi_ref from exact
// difference forms of Eq. 12 in rho - rho_ref and T - T_ref, so that neighbour
// differences in the force keep their low-order bits.
// PAIRED (FP32 thermal, interior path): the two sums of Eqs. 4 and 17 in the two lanes of
// paired FP32 additions (same association, each lane rounded as before).
template <typename Real, bool THERMAL, bool PAIRED = false>
__device__ __forceinline__ NodeState<Real> node_state(const Real (&fc)[9], const Real (&gc)[9],
                                                      const KConst<Real>& C, bool multiphase, bool hazi = false) {
  NodeState<Real> o;
  o.hmc = Real(0);
  const Real rho_ref = C.rho_ref;
  Real sum_g = Real(0);
  if constexpr (PAIRED && THERMAL && sizeof(Real) == 4) {
    float2 q[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) q[i] = make_float2(fc[i], gc[i]);
    const float2 sum = __fadd2_rn(__fadd2_rn(__fadd2_rn(__fadd2_rn(q[0], q[1]), __fadd2_rn(q[2], q[3])),
                                             __fadd2_rn(__fadd2_rn(q[4], q[5]), __fadd2_rn(q[6], q[7]))),
                                  q[8]);
    o.drho = sum.x;
    sum_g = sum.y;
  } else {
    o.drho = ((fc[0] + fc[1]) + (fc[2] + fc[3])) + ((fc[4] + fc[5]) + (fc[6] + fc[7])) + fc[8];
    if (THERMAL) sum_g = ((gc[0] + gc[1]) + (gc[2] + gc[3])) + ((gc[4] + gc[5]) + (gc[6] + gc[7])) + gc[8];
  }
  o.rho = rho_ref + o.drho;
  const Real jx = (fc[1] - fc[3]) + (fc[5] - fc[6]) + (fc[8] - fc[7]);
  const Real jy = (fc[2] - fc[4]) + (fc[5] + fc[6]) - (fc[7] + fc[8]);
  const Real inv_rho = fast_rcp(o.rho);
  o.inv_rho = inv_rho;
  o.ux = jx * inv_rho;
  o.uy = jy * inv_rho;
  if (THERMAL) {
    o.dT = sum_g;
    o.T = C.T_ref + o.dT;
  } else {
    o.dT = Real(0);
    o.T = C.T0;
  }
  o.dpsi = Real(0);
  o.p = o.rho * Real(1.0 / 3.0);
  o.coef = Real(0);
  Real dpdT = Real(0);
  bool bad = !(o.rho > Real(0));
  if (multiphase) {
    const Real pa = C.a, pb = C.b, pR = C.R, kappa = C.kappa, inv_sqrtTc = C.inv_sqrtTc;
    const Real rho_c = o.rho, drho_c = o.drho, T_c = o.T, dT_c = o.dT;
    const Real br = pb * rho_c;
    const Real inv1 = fast_rcp(Real(1) - br);
    const Real invD = fast_rcp(Real(1) + br * (Real(2) - br));
    const Real rr_den = rho_c * rho_c * invD;
    Real alpha, sa = Real(0), inv_sT = Real(0), sT = Real(0);
    if (THERMAL) {
      inv_sT = fast_rsqrt(T_c);
      sT = T_c * inv_sT;
      sa = Real(1) + kappa * (Real(1) - sT * inv_sqrtTc);
      alpha = sa * sa;
    } else {
      alpha = C.alpha0;
    }
    Real rad;
    if (sizeof(Real) == 4) {
      const Real rr = rho_ref;
      // R (rho T / (1 - b rho) - rho_ref T_ref / (1 - b rho_ref)) and the attraction term's
      // difference, as exact difference forms in drho = rho - rho_ref and dT = T - T_ref
      const Real dA = C.R_u1r * (drho_c * T_c * inv1 + (THERMAL ? rr * dT_c : Real(0)));
      Real dB = C.a_Dr * alpha * drho_c * (rho_c + rr + C.twob_rr * rho_c) * invD;
      if (THERMAL) {
        const Real dsa = C.nk_sTc * dT_c * fast_rcp(sT + C.sqrtT_r);
        dB += C.a_rr2_Dr * dsa * (sa + C.sa_r);
      }
      const Real dp = dA - dB;
      const Real drad = (dp - drho_c * Real(1.0 / 3.0)) * C.psi_scale;
      rad = C.rad_ref + drad;
      const Real psi = fast_sqrt(fmax(rad, Real(0)));
      const Real den = psi + C.psi_ref;
      o.dpsi = den > Real(0) ? drad * fast_rcp(den) : Real(0);
      o.p = C.p_ref + dp;
    } else {
      o.p = rho_c * pR * T_c * inv1 - pa * alpha * rr_den;
      rad = (o.p - rho_c * Real(1.0 / 3.0)) * C.psi_scale;
      o.dpsi = fast_sqrt(fmax(rad, Real(0)));
    }
    bad = bad || !(br < Real(1)) || !(rad >= Real(0));
    if (THERMAL) {
      const Real dalpha = C.nk_sTc * sa * inv_sT;  // d alpha / dT = -kappa sqrt(alpha) / sqrt(T Tc)
      dpdT = rho_c * pR * inv1 - pa * dalpha * rr_den;
    }
  }
  if (THERMAL) {
    bad = bad || !isfinite(o.T);
    if (hazi) {  // first Eq. 19: T div u + T (dp/dT)_rho / (rho^2 c_v) drho/dt
      o.coef = o.T;
      o.hmc = o.T * dpdT * inv_rho * inv_rho * C.inv_cv;
    } else {     // second Eq. 19
      o.coef = o.T * (Real(1) - dpdT * inv_rho * C.inv_cv);
    }
  }
  o.bad = bad;
  return o;
}

// Interaction force of Eqs. 9, 10, 14, 15 from the neighbours' d = psi - psi_ref
// (d = 0 for solid neighbours).  With psi = psi_ref + d the beta-mixed sums reduce to
// F = -(psi_ref + beta d_c) t1 - (1 - beta)/2 t2, t1 = sum G_i d_i c_i,
// t2 = sum G_i d_i^2 c_i, plus the wall rows' reference parts with Eq. 15.
template <typename Real>
__device__ __forceinline__ void sc_force(Real dc, Real dE, Real dW, Real dN, Real dNE, Real dNW, Real dS, Real dSE,
                                         Real dSW, bool sol_m, bool sol_p, const KConst<Real>& C, Real& Fx,
                                         Real& Fy) {
  const Real G2 = C.G2, Gh = C.Gh;
  const Real t1x = G2 * (dE - dW) + Gh * ((dNE - dNW) + (dSE - dSW));
  const Real t1y = G2 * (dN - dS) + Gh * ((dNE + dNW) - (dSE + dSW));
  const Real t2x = G2 * (dE - dW) * (dE + dW) + Gh * ((dNE - dNW) * (dNE + dNW) + (dSE - dSW) * (dSE + dSW));
  const Real t2y = G2 * (dN - dS) * (dN + dS) + Gh * ((dNE - dSE) * (dNE + dSE) + (dNW - dSW) * (dNW + dSW));
  const Real lead = C.psi_ref + C.beta * dc;
  Fx = -lead * t1x - C.mix * t2x;
  Fy = -lead * t1y - C.mix * t2y;
  if (sol_m) Fy += C.wall0 + dc * C.wall1;
  if (sol_p) Fy -= C.wall0 + dc * C.wall1;
}

// FP32 form of sc_force for the interior path, with paired FP32 instructions: the x and y
// components in the two lanes of a register pair, and the diagonal neighbours' sums and
// differences formed two at a time.  The same expressions as sc_force (the products keep its
// difference-of-squares form (a - b)(a + b)); only the grouping of the roundings differs.
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }

__device__ __forceinline__ void sc_force_paired(float dc, float dE, float dW, float dN, float dNE, float dNW, float dS,
                                                float dSE, float dSW, bool sol_m, bool sol_p, const KConst<float>& C,
                                                float& Fx, float& Fy) {
  const float2 P = make_float2(dE, dN), Q = make_float2(dW, dS);
  const float2 A = f2sub(P, Q), S = __fadd2_rn(P, Q);        // (dE - dW, dN - dS), (dE + dW, dN + dS)
  const float2 U = make_float2(dNE, dSE), V = make_float2(dNW, dSW);
  const float2 m = f2sub(U, V), p = __fadd2_rn(U, V);        // (dNE - dNW, dSE - dSW), (dNE + dNW, dSE + dSW)
  const float2 U2 = make_float2(dNE, dNW), V2 = make_float2(dSE, dSW);
  const float2 b = f2sub(U2, V2), a = __fadd2_rn(U2, V2);    // (dNE - dSE, dNW - dSW), (dNE + dSE, dNW + dSW)
  const float2 mp = __fmul2_rn(m, p), ab = __fmul2_rn(b, a);
  const float2 G2 = make_float2(C.G2, C.G2), Gh = make_float2(C.Gh, C.Gh);
  const float2 t1 = __ffma2_rn(G2, A, __fmul2_rn(Gh, make_float2(m.x + m.y, p.x - p.y)));
  const float2 t2 = __ffma2_rn(__fmul2_rn(G2, A), S, __fmul2_rn(Gh, make_float2(mp.x + mp.y, ab.x + ab.y)));
  const float nlead = -(C.psi_ref + C.beta * dc);
  const float2 F = __ffma2_rn(make_float2(nlead, nlead), t1, __fmul2_rn(make_float2(-C.mix, -C.mix), t2));
  Fx = F.x;
  Fy = F.y;
  if (sol_m) Fy += C.wall0 + dc * C.wall1;
  if (sol_p) Fy -= C.wall0 + dc * C.wall1;
}

// The 9 staged populations of one node, population i at p[i * stride].
template <typename Real>
struct StridedPops {
  const Real* p;
  int stride;
  __device__ __forceinline__ Real operator()(int i) const { return p[i * stride]; }
};

// Population i of one node in an output buffer: p[i * plane] (p at the node in plane 0).
template <typename Real>
struct PlaneOut {
  Real* p;
  int plane;
  __device__ __forceinline__ Real& operator()(int i) const { return p[i * plane]; }
};
#ifdef LBM_BOUNDS_CHECK
// PlaneOut of the bounds-checked build: element m + i * plane of a buffer of n elements.
template <typename Real>
struct CheckedPlaneOut {
  Real* base;
  int m, plane;
  InstState* st;
  long long n;
  __device__ __forceinline__ Real& operator()(int i) const {
    const long long k = (long long)m + (long long)i * plane;
    return idx_ok(st, k, n) ? base[k] : bounds_sink<Real>();
  }
};
#endif
// Output view of node m (element index in plane 0) of a 9-plane buffer `base` of n elements.
template <typename Real>
__device__ __forceinline__ auto plane_out(Real* base, int m, int plane, InstState* st, long long n) {
#ifdef LBM_BOUNDS_CHECK
  return CheckedPlaneOut<Real>{base, m, plane, st, n};
#else
  (void)st;
  (void)n;
  return PlaneOut<Real>{base + m, plane};
#endif
}
// The same through the descriptor's plane offsets: base[m + poff[i]], m the node's element
// index (one add per population, the offsets read from the descriptor).
template <typename Real>
struct OffsetOut {
  Real* base;
  int m;
  const Inst& I;
  __device__ __forceinline__ Real& operator()(int i) const {
#ifdef LBM_BOUNDS_CHECK
    const int k = m + I.poff[i];
    return idx_ok(I.st, k, 9 * I.plane) ? base[k] : bounds_sink<Real>();
#else
    return base[m + I.poff[i]];
#endif
  }
};

// BGK toward f^eq(rho, u_eq) (Eqs. 2-3) plus the exact-difference term (Eq. 5),
// written pairwise over opposite directions i, i': with cu = c_i.u, cd = c_i.du and
// cs = c_i.(2u + du), omega f^eq_i + F_i = w_i (K + 4.5 rho (omega cu^2 + cd cs))
// + 3 w_i rho (omega cu + cd), K = omega (drho - 1.5 rho u.u) - 1.5 rho du.(2u + du);
// the direction i' flips the sign of the second term only.  fs(i): the pulled
// population i of the node; fo(i): population i of the node in the output buffer.
template <typename Real, typename Pops, typename Out>
__device__ __forceinline__ void collide_f(const Pops& fs, const Out& fo, Real rho,
                                          Real drho, Real ux, Real uy, Real dux, Real duy, Real omega_f) {
  const Real sx = Real(2) * ux + dux, sy = Real(2) * uy + duy;
  const Real usq = ux * ux + uy * uy;
  const Real K = omega_f * (drho - Real(1.5) * rho * usq) - Real(1.5) * rho * (dux * sx + duy * sy);
  const Real r45 = Real(4.5) * rho, r3 = Real(3) * rho, keep = Real(1) - omega_f;
  auto pair = [&](int i, int j, Real cu, Real cd, Real cs, Real w) {
    const Real sym = w * (K + r45 * (omega_f * cu * cu + cd * cs));
    const Real anti = w * r3 * (omega_f * cu + cd);
    fo(i) = keep * fs(i) + sym + anti;
    fo(j) = keep * fs(j) + sym - anti;
  };
  fo(0) = keep * fs(0) + lat_w<Real>(0) * K;
  pair(1, 3, ux, dux, sx, lat_w<Real>(1));
  pair(2, 4, uy, duy, sy, lat_w<Real>(2));
  pair(5, 7, ux + uy, dux + duy, sx + sy, lat_w<Real>(5));
  pair(6, 8, uy - ux, duy - dux, sy - sx, lat_w<Real>(6));
}

// Eq. 16 with g^eq of Eq. 18 and the source phi (second Eq. 19), pairwise as for f:
// omega g^eq_i + w_i phi = w_i (Kg + 4.5 omega T cu^2) + 3 w_i omega T cu.
template <typename Real, typename Pops, typename Out>
__device__ __forceinline__ void collide_g(const Pops& gs, const Out& go, Real T,
                                          Real dT, Real uax, Real uay, Real phi, Real omega_g) {
  const Real usq = uax * uax + uay * uay;
  const Real Kg = omega_g * (dT - Real(1.5) * T * usq) + phi;
  const Real t45 = Real(4.5) * omega_g * T, t3 = Real(3) * omega_g * T, keep = Real(1) - omega_g;
  auto pair = [&](int i, int j, Real cu, Real w) {
    const Real sym = w * (Kg + t45 * cu * cu);
    const Real anti = w * t3 * cu;
    go(i) = keep * gs(i) + sym + anti;
    go(j) = keep * gs(j) + sym - anti;
  };
  go(0) = keep * gs(0) + lat_w<Real>(0) * Kg;
  pair(1, 3, uax, lat_w<Real>(1));
  pair(2, 4, uay, lat_w<Real>(2));
  pair(5, 7, uax + uay, lat_w<Real>(5));
  pair(6, 8, uay - uax, lat_w<Real>(6));
}

// FP32 forms of the two collisions for the interior path, with paired FP32 arithmetic
// (FADD2 / FMUL2 / FFMA2: two independent operations per instruction).  The pairs of
// opposite directions that share a weight are computed two at a time: the axis pairs
// (1,3) and (2,4) in the two lanes of one register pair, the diagonal pairs (5,7) and (6,8)
// in another.  Same formulas as collide_f / collide_g; only the grouping of the roundings
// differs (paired instructions round each lane exactly as the scalar instruction would).
__device__ __forceinline__ float2 f2bc(float a) { return make_float2(a, a); }

template <typename Pops, typename Out>
__device__ __forceinline__ void collide_f_paired(const Pops& fs, const Out& fo, float rho, float drho, float ux,
                                                 float uy, float dux, float duy, float omega_f) {
  constexpr float w0 = LatWeights<float>::w0(), w1 = LatWeights<float>::w1(), w5 = LatWeights<float>::w5();
  const float2 U = make_float2(ux, uy), D = make_float2(dux, duy);
  const float2 S = __ffma2_rn(f2bc(2.0f), U, D);  // (2u + du) per axis
  const float2 UU = __fmul2_rn(U, U);
  const float2 DS = __fmul2_rn(D, S);
  const float r15 = 1.5f * rho;
  const float K = omega_f * (drho - r15 * (UU.x + UU.y)) - r15 * (DS.x + DS.y);
  const float r45 = 4.5f * rho, r3 = 3.0f * rho, keep = 1.0f - omega_f;
  fo(0) = keep * fs(0) + w0 * K;
  const float2 KEEP = f2bc(keep), R45 = f2bc(r45), KK = f2bc(K), WF = f2bc(omega_f), NEG = f2bc(-1.0f);
  auto pairs = [&](float2 cu, float2 cd, float2 cs, float w, int i, int j, int ib, int jb) {
    const float2 wcu = __fmul2_rn(WF, cu);                                     // omega c.u
    const float2 X = __ffma2_rn(wcu, cu, __fmul2_rn(cd, cs));                  // omega cu^2 + cd cs
    const float2 sym = __fmul2_rn(f2bc(w), __ffma2_rn(R45, X, KK));           // w (K + 4.5 rho X)
    const float2 anti = __fmul2_rn(f2bc(w * r3), __fadd2_rn(wcu, cd));        // 3 w rho (omega cu + cd)
    const float2 plus = __fadd2_rn(sym, anti), minus = __ffma2_rn(anti, NEG, sym);
    const float2 a = __ffma2_rn(KEEP, make_float2(fs(i), fs(j)), plus);
    const float2 b = __ffma2_rn(KEEP, make_float2(fs(ib), fs(jb)), minus);
    fo(i) = a.x;
    fo(j) = a.y;
    fo(ib) = b.x;
    fo(jb) = b.y;
  };
  pairs(U, D, S, w1, 1, 2, 3, 4);  // lanes: (1,3) with c.u = ux, (2,4) with c.u = uy
  const float2 PM = make_float2(1.0f, -1.0f);
  const float2 Ud = __ffma2_rn(f2bc(ux), PM, f2bc(uy));    // (ux + uy, uy - ux)
  const float2 Dd = __ffma2_rn(f2bc(dux), PM, f2bc(duy));
  const float2 Sd = __ffma2_rn(f2bc(S.x), PM, f2bc(S.y));
  pairs(Ud, Dd, Sd, w5, 5, 6, 7, 8);  // lanes: (5,7) with c.u = ux + uy, (6,8) with c.u = uy - ux
}

template <typename Pops, typename Out>
__device__ __forceinline__ void collide_g_paired(const Pops& gs, const Out& go, float T, float dT, float uax,
                                                 float uay, float phi, float omega_g) {
  constexpr float w0 = LatWeights<float>::w0(), w1 = LatWeights<float>::w1(), w5 = LatWeights<float>::w5();
  const float2 U = make_float2(uax, uay);
  const float2 UU = __fmul2_rn(U, U);
  const float Kg = omega_g * (dT - 1.5f * T * (UU.x + UU.y)) + phi;
  const float t45 = 4.5f * omega_g * T, t3 = 3.0f * omega_g * T, keep = 1.0f - omega_g;
  go(0) = keep * gs(0) + w0 * Kg;
  const float2 KEEP = f2bc(keep), NEG = f2bc(-1.0f);
  auto pairs = [&](float2 cu, float w, int i, int j, int ib, int jb) {
    const float2 sym = __ffma2_rn(f2bc(w * t45), __fmul2_rn(cu, cu), f2bc(w * Kg));  // w (Kg + 4.5 omega T cu^2)
    const float2 anti = __fmul2_rn(f2bc(w * t3), cu);                                 // 3 w omega T cu
    const float2 plus = __fadd2_rn(sym, anti), minus = __ffma2_rn(anti, NEG, sym);
    const float2 a = __ffma2_rn(KEEP, make_float2(gs(i), gs(j)), plus);
    const float2 b = __ffma2_rn(KEEP, make_float2(gs(ib), gs(jb)), minus);
    go(i) = a.x;
    go(j) = a.y;
    go(ib) = b.x;
    go(jb) = b.y;
  };
  pairs(U, w1, 1, 2, 3, 4);
  pairs(__ffma2_rn(f2bc(uax), make_float2(1.0f, -1.0f), f2bc(uay)), w5, 5, 6, 7, 8);
}

// Issue the asynchronous pull of one node's populations into f_dst/g_dst (stride
// dstride).  Interior links copy f*_i(x - c_i); links from a wall row copy
// f*_opp(x) (halfway bounce-back; boundary_fill applies the g sign flip and wall
// temperature); links from outside an open end are left for boundary_fill.
template <typename Real, bool THERMAL>
__device__ __forceinline__ void pull_node(Real* f_dst, Real* g_dst, int dstride, const Real* __restrict__ Fin,
                                          const Real* __restrict__ Gin, int plane, int pitch, int xn, int rn,
                                          int nx, int ny, bool perx, bool pery, bool local, const NodeBC& nb,
                                          InstState* bst) {
  const int node = rn * pitch + xn;
  const long long nbuf = 9LL * plane;  // elements of one population buffer (bounds checks)
  if (local) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      if (!idx_ok(bst, node + i * plane, nbuf)) continue;
      cp_async_elem(f_dst + i * dstride, Fin + node + i * plane);
      if (THERMAL) cp_async_elem(g_dst + i * dstride, Gin + node + i * plane);
    }
    return;
  }
  if (xn >= 1 && xn <= nx - 2 && rn >= 1 && rn <= ny - 2) {
    // interior: the source of link i is node - c_iy * pitch - c_ix in plane i
    const Real* fn = Fin + node;
    const Real* gn = Gin + node;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int off = i * plane - lat_cy(i) * pitch - lat_cx(i);
      if (!idx_ok(bst, node + off, nbuf)) continue;
      cp_async_elem(f_dst + i * dstride, fn + off);
      if (THERMAL) cp_async_elem(g_dst + i * dstride, gn + off);
    }
    return;
  }
  int xm = xn - 1, xp = xn + 1, rm = rn - 1, rp = rn + 1;
  if (perx) {
    if (xm < 0) xm += nx;
    if (xp >= nx) xp -= nx;
  }
  if (pery) {
    if (rm < 0) rm += ny;
    if (rp >= ny) rp -= ny;
  }
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int cxi = lat_cx(i), cyi = lat_cy(i);
    const bool wall = (cyi == 1 && nb.wlo) || (cyi == -1 && nb.whi);
    const bool unknown = (cxi == 1 && nb.inl) || (cxi == -1 && nb.outl) || (cyi == -1 && nb.top);
    int src;
    int pl = i;
    if (wall) {
      src = node;
      pl = lat_opp(i);
    } else if (!unknown) {
      src = (cyi == 1 ? rm : (cyi == -1 ? rp : rn)) * pitch + (cxi == 1 ? xm : (cxi == -1 ? xp : xn));
    } else {
      continue;
    }
    if (!idx_ok(bst, pl * plane + src, nbuf)) continue;
    cp_async_elem(f_dst + i * dstride, Fin + pl * plane + src);
    if (THERMAL) cp_async_elem(g_dst + i * dstride, Gin + pl * plane + src);
  }
}

// Completion of a launch by the tile drawing its last ticket: the diagnostics record
// of the step, the domain-mean density for the next step's buoyancy, and the step
// counter (tot: the launch's totals of deviations from the storage references).
template <bool THERMAL, int MODE>
__device__ __forceinline__ void finish_step(const Inst& I, InstState* st, const double (&tot)[NPART],
                                            long long step) {
  const double n = (double)I.nx * (double)I.ny;
  const double mass = tot[0] + n * I.rho_ref;
  const double energy = THERMAL ? tot[1] + n * I.T_ref : n * I.T0;
  const bool channel = I.geometry == GEOM_CHANNEL;
  if (MODE == MODE_STEP) {
    double dtstar = 0.0;
    const bool heat_now = THERMAL && I.heater_len > 0 && step >= I.heat_on_step && I.geometry != GEOM_PERIODIC;
    if (heat_now) {
      const int hx0 = I.heater_x0, hx1 = I.heater_x0 + I.heater_len;
      const int lo = hx0 < 0 ? 0 : hx0, hi = hx1 > I.nx ? I.nx : hx1;
      if (hi > lo) {
        const double tnb = tot[2] / (double)(hi - lo) + I.T_ref;
        dtstar = (I.T_heat - tnb) / (I.T_heat - energy / n);
      }
    }
    double* rec = I.ring + (step % RING) * NDIAG;
    rec[0] = (double)step;
    rec[1] = mass;
    rec[2] = energy;
    rec[3] = mass / n;
    rec[4] = channel ? __ldcg(&st->p_probe[2 * (step & 1)]) - __ldcg(&st->p_probe[2 * (step & 1) + 1]) : 0.0;
    rec[5] = dtstar;
    rec[6] = channel ? tot[3] : 0.0;
    rec[7] = channel ? tot[4] : 0.0;
    rec[8] = tot[5];
    rec[9] = tot[6];
    rec[10] = tot[7];
    rec[11] = tot[8];
    st->rho_avg[step & 1] = mass / n;
    st->local_read = 0;
  } else {
    st->rho_avg[(step - 1) & 1] = mass / n;
  }
  // every tile of this step has read the open-end mass of the step before (its slot is free
  // until step + 3 posts there), and has taken its ticket
  st->counter[step & 1] = 0u;
  st->open_mass[(step - 1) & 3] = 0;
  st->open_posted[(step - 1) & 3] = 0u;
  if (MODE == MODE_STEP) {
    __threadfence();  // the record, the mean and the resets are visible before the step count
    atomicExch(reinterpret_cast<unsigned long long*>(&st->step), (unsigned long long)(step + 1));
  }
}

// End of a tile of a MODE_STEP / MODE_MOMENTS launch: post its partial sums (acc, per thread).
// The tile's FP64 sums (warp shuffles, then warps in order) are rounded to the fixed-point
// totals' grid and added to them by NPART integer atomics; then a ticket counts the tile.  The
// tile drawing the last ticket takes the totals (and leaves zeros for the next launch) by one
// atomic exchange each and finishes the step.  A sum outside the totals' range (only a diverged
// run, or a NaN) marks the instance unstable.  Every tile of a launch must post exactly once.
// open: the tile also posts open_acc, its share of the mass that this step's pull took in and
// let out through the channel's open ends (the overlapped persistent loop derives the next
// step's buoyancy mean from it); the fixed-point grid is the inflow total's.  NA: the partials
// the tile can have nonzero (the first NA of acc; an interior tile has mass, energy and the
// heater row only); a total that a tile leaves at zero takes no atomic.
template <int BLOCK, bool THERMAL, int MODE, int NA = NPART>
__device__ __forceinline__ void post_partials(const Inst& I, InstState* st, const Tile& tile, const double (&acc)[NPART],
                                              double (*red)[NPART], int* flag, long long step, bool open = false,
                                              double open_acc = 0.0) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned long long* const sums = I.sums + (step & 1) * NPART;
#pragma unroll
  for (int j = 0; j < NA; ++j) {
    double x = acc[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp][j] = x;
  }
  if (open) {
    double x = open_acc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    __shared__ double s_open[BLOCK / 32];
    if (lane == 0) s_open[warp] = x;
    __syncthreads();
    if (tid == 0) {
      double sum = 0.0;
      for (int w = 0; w < BLOCK / 32; ++w) sum += s_open[w];
      const double q = sum * I.fix_scale[3];
      long long v = 0;
      if (fabs(q) < 0x1p62) v = __double2ll_rn(q);
      else atomicOr(&st->status, STATUS_UNSTABLE);
      atomicAdd(reinterpret_cast<unsigned long long*>(&st->open_mass[step & 3]), (unsigned long long)v);
      __threadfence();  // the addition is performed before the count
      atomicAdd(&st->open_posted[step & 3], 1u);
    }
  }
  __syncthreads();
  if (tid < NA) {
    double sum = 0.0;
    for (int w = 0; w < BLOCK / 32; ++w) sum += red[w][tid];
    const double x = sum * I.fix_scale[tid];  // a power of two: exact
    long long q = 0;
    if (fabs(x) < 0x1p62) q = __double2ll_rn(x);
    else atomicOr(&st->status, STATUS_UNSTABLE);
    if (q != 0) atomicAdd(sums + tid, (unsigned long long)q);
  }
  __syncthreads();
  if (tid == 0) {
    __threadfence();  // the block's additions are performed before its ticket
    const unsigned ticket = atomicAdd(&st->counter[step & 1], 1u);
    *flag = (ticket == (unsigned)(tile.ntiles - 1));
  }
  __syncthreads();
  if (!*flag) return;
  __threadfence();
  if (tid < NPART) red[0][tid] = (double)(long long)atomicExch(sums + tid, 0ull) * I.fix_unscale[tid];
  __syncthreads();
  if (tid == 0) {
    double tot[NPART];
#pragma unroll
    for (int j = 0; j < NPART; ++j) tot[j] = red[0][j];
    finish_step<THERMAL, MODE>(I, st, tot, step);
  }
}

// ---------------------------------------------------------------------------
// Interior path of the step (MODE_STEP, lean form).  A tile whose pulled columns
// [x0 - 2, x0 + B - 6) all lie in [1, nx - 2] of a channel or walls lattice meets no open
// end and no wrap in x, so its nodes need none of the general loop's per-node boundary
// logic: a pull is one add per link (the descriptor's link offsets), the stencil
// neighbours are the adjacent lanes, and only the wall rows 0 and ny - 1 take the wall
// branches (bounce-back links, anti-bounce-back temperature, solid neighbours of the force,
// one-sided wall divergence), decided once per row for the whole CTA.  The arithmetic is the
// general loop's, expression for expression, so the results are bit-identical to it.
// ---------------------------------------------------------------------------

// Anti-bounce-back of g on the links of a wall row (the wall part of boundary_fill): the
// links with c_y = +1 come from the bottom wall (lo), those with c_y = -1 from the top (hi).
template <typename Real>
__device__ __forceinline__ void wall_temperature(Real (&gc)[9], bool lo, bool hi, int xn, const Inst& I,
                                                 const KConst<Real>& C, long long step) {
  const bool heat_bc = I.heater_len > 0 && (step - 1) >= I.heat_on_step;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int cxi = lat_cx(i), cyi = lat_cy(i);
    if ((cyi == 1 && lo) || (cyi == -1 && hi)) {
      Real dTw = C.dT_in;
      if (cyi == 1 && heat_bc) {
        const int sx = xn - cxi;
        if (sx >= I.heater_x0 && sx < I.heater_x0 + I.heater_len) dTw = C.dT_heat;
      }
      gc[i] = -gc[i] + Real(2) * lat_w<Real>(i) * dTw;
    }
  }
}

// Shared memory (smem, interior_smem_bytes): per-thread rings of the staged f (FI_SLOTS rows)
// and g (GI_SLOTS rows), then three-row rings of psi, u_act,x and u_act,y.  Each row's pull is
// issued LOOKAHEAD iterations before it is used.
template <typename Real, bool THERMAL, int B>
__device__ __forceinline__ void interior_rows(const Inst& I, const KConst<Real>& C, Real rra, const Tile& tile,
                                              long long step, bool local, unsigned char* smem, Real& acc_m,
                                              Real& acc_e, Real& acc_h, bool& bad_any) {
  constexpr int W = out_cols<B>();
  constexpr int NS = B - 4;
  Real* const sF = reinterpret_cast<Real*>(smem);           // [FI_SLOTS][9][NS]
  Real* const sG = sF + FI_SLOTS * 9 * NS;                   // [GI_SLOTS][9][NS]
  Real* const sPsi = sG + (THERMAL ? GI_SLOTS * 9 * NS : 0);  // [3][NS]
  Real* const sUx = sPsi + 3 * NS;                           // [3][NS]
  Real* const sUy = sUx + 3 * NS;                            // [3][NS]
  const int tid = threadIdx.x;
  const bool act = tid < NS;
  const int s = act ? tid : 0;
  const int xn = tile.x0 - 2 + s;
  const bool out_col = act && s >= 2 && s < W + 2;
  const bool f_col = act && s >= 1 && s <= W + 2;
  const int ny = I.ny, pitch = I.pitch;
  const int y0 = tile.y0, y1 = tile.y1;
  const int kend = y1 - y0 + 4;
  const bool multiphase = I.multiphase != 0;
  const bool heat_col = xn >= I.heater_x0 && xn < I.heater_x0 + I.heater_len;
  const Real* __restrict__ Fin = static_cast<const Real*>(I.f[step & 1]);
  const Real* __restrict__ Gin = static_cast<const Real*>(I.g[step & 1]);
  Real* __restrict__ Fout = static_cast<Real*>(I.f[(step + 1) & 1]);
  Real* __restrict__ Gout = static_cast<Real*>(I.g[(step + 1) & 1]);

  // pull of row y0 - 2 + k into ring slots (fslot, gslot): interior rows take each link from
  // node + loff[i]; a wall row takes its wall links from the node's own opposite population
  // (halfway bounce-back); right after an initialisation every node copies its own populations
  auto issue_row = [&](int k, int fslot, int gslot) {
    const int rr = y0 - 2 + k;
    if (act && k < kend && rr >= 0 && rr < ny) {
      Real* fd = sF + fslot * 9 * NS + s;
      Real* gd = sG + gslot * 9 * NS + s;
      const int node = rr * pitch + xn;
      const long long nbuf = 9LL * I.plane;  // elements of one population buffer (bounds checks)
      if (local) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          const int src = node + I.poff[i];
          if (!idx_ok(I.st, src, nbuf)) continue;
          cp_async_elem(fd + i * NS, Fin + src);
          if (THERMAL) cp_async_elem(gd + i * NS, Gin + src);
        }
      } else if (rr > 0 && rr < ny - 1) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          const int src = node + I.loff[i];
          if (!idx_ok(I.st, src, nbuf)) continue;
          cp_async_elem(fd + i * NS, Fin + src);
          if (THERMAL) cp_async_elem(gd + i * NS, Gin + src);
        }
      } else {
        const bool lo = rr == 0, hi = rr == ny - 1;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          const int cyi = lat_cy(i);
          const bool wall = (cyi == 1 && lo) || (cyi == -1 && hi);
          const int src = wall ? node + I.poff[lat_opp(i)] : node + I.loff[i];
          if (!idx_ok(I.st, src, nbuf)) continue;
          cp_async_elem(fd + i * NS, Fin + src);
          if (THERMAL) cp_async_elem(gd + i * NS, Gin + src);
        }
      }
    }
    cp_async_commit();
  };

  Real rho_p = Real(1), drho_p = Real(0), ux_p = Real(0), uy_p = Real(0), T_p = C.T0, dT_p = Real(0), coef_p = Real(0);
  Real inv_rho_p = Real(1);
  Real T_p2 = C.T0, dT_p2 = Real(0), coef_p2 = Real(0);
  // ring slots of row r = y0 - 2 + k: f (k mod FI_SLOTS), g (k mod GI_SLOTS), psi and u_act (k mod 3)
  int f_cur = 0, g_cur = 0, p_cur = 0;
#pragma unroll
  for (int a = 0; a < LOOKAHEAD; ++a) issue_row(a, a, a);
  for (int k = 0; k < kend; ++k) {
    const int r = y0 - 2 + k;
    const int f_prev = f_cur == 0 ? FI_SLOTS - 1 : f_cur - 1;                      // row r-1
    const int f_issue = f_cur >= 2 ? f_cur - 2 : f_cur + (FI_SLOTS - 2);            // row r+LOOKAHEAD
    const int g_issue = g_cur >= 3 ? g_cur - 3 : g_cur + (GI_SLOTS - 3);            // row r+LOOKAHEAD
    const int g_prev2 = g_cur >= 2 ? g_cur - 2 : g_cur + (GI_SLOTS - 2);            // row r-2
    const int p_prev = p_cur == 0 ? 2 : p_cur - 1;                 // row r-1
    const int p_prev2 = p_cur == 2 ? 0 : p_cur + 1;                // row r-2 (= r+1 = r-3)
    NodeState<Real> ns;
    ns.rho = Real(1); ns.inv_rho = Real(1); ns.drho = Real(0); ns.ux = Real(0); ns.uy = Real(0);
    ns.T = C.T0; ns.dT = Real(0); ns.coef = Real(0); ns.dpsi = Real(0);
    issue_row(k + LOOKAHEAD, f_issue, g_issue);
    cp_async_wait_lookahead<LOOKAHEAD>();  // this thread's copies of row r have landed

    // ===================== phase A: row r =====================
    if (act && r >= 0 && r < ny) {
      const Real* fs = sF + f_cur * 9 * NS + s;
      Real* gs = sG + g_cur * 9 * NS + s;
      Real fc[9], gc[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        fc[i] = fs[i * NS];
        gc[i] = THERMAL ? gs[i * NS] : Real(0);
      }
      if (THERMAL && !local && (r == 0 || r == ny - 1)) {
        wall_temperature<Real>(gc, r == 0, r == ny - 1, xn, I, C, step);
#pragma unroll
        for (int i = 0; i < 9; ++i) gs[i * NS] = gc[i];
      }
      ns = node_state<Real, THERMAL, true>(fc, gc, C, multiphase, false);
      bad_any = bad_any || ns.bad;
      sPsi[p_cur * NS + s] = ns.dpsi;
      if (out_col && r >= y0 && r < y1) {
        acc_m += ns.drho;
        if (THERMAL) {
          acc_e += ns.dT;
          if (r == 0 && heat_col) acc_h += ns.dT;
        }
      }
    }
    __syncthreads();

    // ===================== phase B: row q = r - 1 =====================
    const int q = r - 1;
    if (f_col && q >= y0 - 1 && q >= 0 && q < ny) {
      Real Fx = Real(0), Fy = Real(0);
      if (multiphase) {
        const Real* P0 = sPsi + p_prev * NS + s;
        const Real* Pp = sPsi + p_cur * NS + s;
        const Real* Pm = sPsi + p_prev2 * NS + s;
        auto force = [&](Real dN, Real dNE, Real dNW, Real dS, Real dSE, Real dSW, bool sol_m, bool sol_p) {
          if constexpr (sizeof(Real) == 4)
            sc_force_paired(P0[0], P0[1], P0[-1], dN, dNE, dNW, dS, dSE, dSW, sol_m, sol_p, C, Fx, Fy);
          else
            sc_force<Real>(P0[0], P0[1], P0[-1], dN, dNE, dNW, dS, dSE, dSW, sol_m, sol_p, C, Fx, Fy);
        };
        if (q > 0 && q < ny - 1) {
          force(Pp[0], Pp[1], Pp[-1], Pm[0], Pm[1], Pm[-1], false, false);
        } else {
          const bool sol_m = q == 0, sol_p = q == ny - 1;  // row q-1 / q+1 is a wall
          force(sol_p ? Real(0) : Pp[0], sol_p ? Real(0) : Pp[1], sol_p ? Real(0) : Pp[-1], sol_m ? Real(0) : Pm[0],
                sol_m ? Real(0) : Pm[1], sol_m ? Real(0) : Pm[-1], sol_m, sol_p);
        }
      }
      Fy -= (drho_p + rra) * C.g_a;  // Eq. 14, gravity along -y
      const Real inv_rho = sizeof(Real) == 8 ? inv_rho_p : fast_rcp(rho_p);
      const Real dux = Fx * inv_rho, duy = Fy * inv_rho;
      const Real uax = ux_p + Real(0.5) * dux, uay = uy_p + Real(0.5) * duy;  // Eq. 7
      sUx[p_prev * NS + s] = uax;
      sUy[p_prev * NS + s] = uay;
      if (out_col && q >= y0 && q < y1) {
        if constexpr (sizeof(Real) == 4)
          collide_f_paired(StridedPops<Real>{sF + f_prev * 9 * NS + s, NS}, OffsetOut<Real>{Fout, q * pitch + xn, I},
                           rho_p, drho_p, ux_p, uy_p, dux, duy, C.omega_f);
        else
          collide_f<Real>(StridedPops<Real>{sF + f_prev * 9 * NS + s, NS}, OffsetOut<Real>{Fout, q * pitch + xn, I},
                          rho_p, drho_p, ux_p, uy_p, dux, duy, C.omega_f);
      }
    }
    __syncthreads();

    // ===================== phase C: row q2 = r - 2 =====================
    if (THERMAL) {
      const int q2 = r - 2;
      if (out_col && q2 >= y0 && q2 < y1) {
        const Real* U2x = sUx + p_prev2 * NS + s;
        const Real* U2y = sUy + p_prev2 * NS + s;
        const Real uxE = U2x[1], uxW = U2x[-1];
        const Real uyN = sUy[p_prev * NS + s];
        const Real uyS = sUy[p_cur * NS + s];  // slot of row r-3
        Real dyu = Real(0.5) * (uyN - uyS);
        if (q2 == 0 || q2 == ny - 1) {  // one-sided wall-normal difference over the fluid rows
          const bool wall_lo = q2 == 0, wall_hi = q2 == ny - 1;
          const Real uyC = U2y[0];
          dyu = (wall_lo && wall_hi) ? Real(0) : (wall_lo ? uyN - uyC : uyC - uyS);
        }
        const Real divu = Real(0.5) * (uxE - uxW) + dyu;
        const Real phi = coef_p2 * divu;
        if constexpr (sizeof(Real) == 4)
          collide_g_paired(StridedPops<Real>{sG + g_prev2 * 9 * NS + s, NS}, OffsetOut<Real>{Gout, q2 * pitch + xn, I},
                           T_p2, dT_p2, U2x[0], U2y[0], phi, C.omega_g);
        else
          collide_g<Real>(StridedPops<Real>{sG + g_prev2 * 9 * NS + s, NS}, OffsetOut<Real>{Gout, q2 * pitch + xn, I},
                          T_p2, dT_p2, U2x[0], U2y[0], phi, C.omega_g);
      }
    }

    T_p2 = T_p;
    dT_p2 = dT_p;
    coef_p2 = coef_p;
    rho_p = ns.rho;
    inv_rho_p = ns.inv_rho;
    drho_p = ns.drho;
    ux_p = ns.ux;
    uy_p = ns.uy;
    T_p = ns.T;
    dT_p = ns.dT;
    coef_p = ns.coef;
    f_cur = f_cur == FI_SLOTS - 1 ? 0 : f_cur + 1;
    g_cur = g_cur == GI_SLOTS - 1 ? 0 : g_cur + 1;
    p_cur = p_cur == 2 ? 0 : p_cur + 1;
  }
}

// ---------------------------------------------------------------------------
// Block form of the fused step.  MODE_STEP advances one step; MODE_FIELDS writes
// rho, u_act and T (FP64) of the current state to the spare f buffer; MODE_POPS
// writes the post-stream populations to the spare buffers; MODE_MOMENTS only
// folds the mean density into the buoyancy slot of the previous step.
// A CTA of B threads owns B - 8 output columns and a band of rows; psi and u_act
// of three rows live in shared rings so that all threads see their neighbours,
// with a barrier after each of phase A (pull, moments, EOS), phase B (force,
// f collision of the row below) and before phase C (g collision two rows below).
// ---------------------------------------------------------------------------
// FULL: the full form, which handles the pool geometry, the Hazi-Markus source and the bubble
// statistics; the lean form (FULL = false, step mode only) compiles them out of the hot loop and
// is launched only for instances that use none of them.
// PCONST: the launch covers one instance whose descriptor and converted constants arrive as
// the kernel parameter kp (read as constant-bank operands instead of shared-memory loads, and
// rematerialised from there instead of held in registers); the buoyancy reference
// rho_ref - rho_avg, which depends on the previous step, is still formed on the device.
// Otherwise every CTA copies its instance's descriptor and constants into shared memory.
// INTERIOR: tiles flagged interior take the interior path (MODE_STEP, lean form only).
//
// A tile's step when the launch, not the instance state, fixes it (the overlapped persistent
// loop): step >= 0 takes step, local and rho_avg_prev (the mean density its buoyancy uses)
// from here, and post_open makes a tile at a channel's inlet or outlet post the mass its pull
// took in and let out there.  The default (step < 0) reads them from the instance state.
struct TileStep {
  long long step = -1;
  bool local = false;
  bool post_open = false;
  double rho_avg_prev = 0.0;
};

// Per-CTA shared state of the step kernels besides the dynamic rings.  Launches over several
// instances also keep the tile's instance descriptor and its converted constants there;
// single-instance launches (PCONST) read both from the kernel parameter.
template <typename Real, int B>
struct StepSharedCommon {
  Real sRra;  // rho_ref - rho_avg of the previous step (buoyancy, Eq. 14)
  double sRed[B / 32][NPART];
  int sLast;
};
template <typename Real, int B, bool PCONST>
struct StepShared : StepSharedCommon<Real, B> {
  Inst sI;
  KConst<Real> sCv;
};
template <typename Real, int B>
struct StepShared<Real, B, true> : StepSharedCommon<Real, B> {};

// The tile's descriptor and constants: the kernel parameter's (PCONST) or the CTA's copies.
template <typename Real, int B, bool PCONST>
__device__ __forceinline__ const Inst& tile_inst(const KParams<Real>& kp, StepShared<Real, B, PCONST>& sh) {
  if constexpr (PCONST) return kp.I;
  else return sh.sI;
}
template <typename Real, int B, bool PCONST>
__device__ __forceinline__ const KConst<Real>& tile_consts(const KParams<Real>& kp, StepShared<Real, B, PCONST>& sh) {
  if constexpr (PCONST) return kp.C;
  else return sh.sCv;
}

// One tile of the fused step (the body of lbm_fused_kernel and of the persistent kernel).
template <typename Real, bool THERMAL, int B, int MODE, bool FULL, bool PCONST, bool INTERIOR>
__device__ __forceinline__ void fused_tile(const Inst* __restrict__ insts, const Tile tile, const KParams<Real>& kp,
                                           unsigned char* dyn_smem, StepShared<Real, B, PCONST>& sh,
                                           const TileStep& ts = TileStep{}) {
  constexpr int BLOCK = B;
  constexpr int W = out_cols<B>();
  constexpr int NS = B - 4;
  Real* const sF = reinterpret_cast<Real*>(dyn_smem);               // [F_SLOTS][9][NS]
  Real* const sG = sF + F_SLOTS * 9 * NS;                           // [G_SLOTS][9][NS]
  Real* const sPsi = sG + (THERMAL ? G_SLOTS * 9 * NS : 0);         // [3][NS]
  Real* const sUx = sPsi + 3 * NS;                                  // [3][NS]
  Real* const sUy = sUx + 3 * NS;                                   // [3][NS]
  Real& sRra = sh.sRra;
  double (*sRed)[NPART] = sh.sRed;
  int& sLast = sh.sLast;

  const int tid = threadIdx.x;
  if constexpr (!PCONST) {
    const int* src = reinterpret_cast<const int*>(insts + tile.inst);
    int* dst = reinterpret_cast<int*>(&sh.sI);
    for (int k = tid; k < (int)(sizeof(Inst) / 4); k += BLOCK) dst[k] = src[k];
    __syncthreads();
  }
  const Inst& I = tile_inst<Real, B, PCONST>(kp, sh);
  InstState* st = I.st;
  const long long step = ts.step >= 0 ? ts.step : st->step;
  if (tid == 0) {
    const double rho_avg_prev = ts.step >= 0 ? ts.rho_avg_prev : st->rho_avg[(step - 1) & 1];
    if constexpr (!PCONST) fill_consts<Real>(sh.sCv, I, rho_avg_prev);
    sRra = Real(I.rho_ref - rho_avg_prev);
  }
  __syncthreads();
  const KConst<Real>& sC = tile_consts<Real, B, PCONST>(kp, sh);

  const int nx = I.nx, ny = I.ny, pitch = I.pitch;
  const int plane = (int)I.plane;  // the host guarantees 9 * plane < 2^31
  const bool local = ts.step >= 0 ? ts.local : st->local_read != 0;
  const bool post_open = MODE == MODE_STEP && ts.post_open && tile.open_end;  // a first step posts 0
  if (INTERIOR && MODE == MODE_STEP && !FULL && tile.interior) {
    Real am = Real(0), ae = Real(0), ah = Real(0);
    bool bad_any = false;
    interior_rows<Real, THERMAL, B>(I, sC, sRra, tile, step, local, dyn_smem, am, ae, ah, bad_any);
    if (bad_any) atomicOr(&st->status, STATUS_UNSTABLE);
    const double acc[NPART] = {(double)am, (double)ae, (double)ah, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    post_partials<BLOCK, THERMAL, MODE, 3>(I, st, tile, acc, sRed, &sLast, step);
    return;
  }
  const bool perx = I.geometry != GEOM_CHANNEL;
  const bool pery = I.geometry == GEOM_PERIODIC;
  const bool channel = I.geometry == GEOM_CHANNEL;
  const bool pool = FULL && I.geometry == GEOM_POOL;
  const bool multiphase = I.multiphase != 0;
  const bool hazi = FULL && THERMAL && I.source_model == 1;
  const bool bubbles = FULL && I.bubble_stats != 0;
  Real* __restrict__ rho_prev = static_cast<Real*>(I.rho_prev);
  const Real* __restrict__ Fin = static_cast<const Real*>(I.f[step & 1]);
  const Real* __restrict__ Gin = static_cast<const Real*>(I.g[step & 1]);
  Real* __restrict__ Fout = static_cast<Real*>(I.f[(step + 1) & 1]);
  Real* __restrict__ Gout = static_cast<Real*>(I.g[(step + 1) & 1]);
  const Real T0 = sC.T0;

  // column owned by this thread: x0 - 2 + tid (two halo columns on each side of the W outputs)
  const int s = tid < NS ? tid : 0;
  const int xc = tile.x0 - 2 + s;
  int xn = xc;
  bool col_ok = tid < NS;
  if (perx) {
    xn = wrap_index(xc, nx);
  } else {
    col_ok = col_ok && xc >= 0 && xc < nx;
  }
  const bool out_col = tid >= 2 && tid < W + 2 && xc < nx;
  const bool f_col = col_ok && s >= 1 && s <= W + 2;
  // shared-memory neighbours; at the open ends the ghost column repeats the end column
  const int sm = (!perx && xc == 0) ? s : s - 1;
  const int sp = (!perx && xc == nx - 1) ? s : s + 1;
  const bool inl = channel && xn == 0;
  const bool outl = channel && xn == nx - 1;

  const int nrow = tile.y1 - tile.y0;
  const int kbeg = (MODE == MODE_STEP) ? 0 : (MODE == MODE_FIELDS ? 1 : 2);
  const int kend = (MODE == MODE_STEP) ? nrow + 4 : (MODE == MODE_FIELDS ? nrow + 3 : nrow + 2);

  auto issue_row = [&](int k, int fslot, int gslot) {
    if (col_ok && k < kend) {
      const int r = tile.y0 - 2 + k;
      if (pery || (r >= 0 && r < ny)) {
        const int rn = pery ? wrap_index(r, ny) : r;
        const NodeBC nb{!pery && rn == 0, !pery && !pool && rn == ny - 1, inl, outl, pool && rn == ny - 1};
        pull_node<Real, THERMAL>(sF + fslot * 9 * NS + s, sG + gslot * 9 * NS + s, NS, Fin, Gin, plane, pitch, xn,
                                 rn, nx, ny, perx, pery, local, nb, I.st);
      }
    }
    cp_async_commit();
  };

  Real acc_m = Real(0), acc_e = Real(0), acc_h = Real(0), acc_fi = Real(0), acc_fo = Real(0);
  float acc_va = 0.0f, acc_wv = 0.0f, acc_hv = 0.0f, acc_zv = 0.0f;  // vapour node counts (exact in FP32)
  double acc_open = 0.0;  // mass through the open ends (post_open)
  const bool zone_col = xn >= I.heater_x0 - I.heater_len && xn < I.heater_x0 + 2 * I.heater_len;
  // node scalars carried between iterations: row r-1 (f collision), row r-2 (g collision)
  Real rho_p = Real(1), drho_p = Real(0), ux_p = Real(0), uy_p = Real(0), T_p = T0, dT_p = Real(0), coef_p = Real(0);
  Real inv_rho_p = Real(1);
  Real T_p2 = T0, dT_p2 = Real(0), coef_p2 = Real(0);
  Real hm_p = Real(0), hm_p2 = Real(0);  // Hazi-Markus source term of rows r-1 and r-2

  // ring slots: f and psi/u rings have 3 slots (row index mod 3), g has 4 (mod 4)
  int f_cur = kbeg % F_SLOTS, g_cur = kbeg % G_SLOTS;
  issue_row(kbeg, f_cur, g_cur);
  for (int k = kbeg; k < kend; ++k) {
    const int r = tile.y0 - 2 + k;
    const int f_next = (f_cur == F_SLOTS - 1) ? 0 : f_cur + 1;
    const int f_prev = (f_cur == 0) ? F_SLOTS - 1 : f_cur - 1;      // row r-1
    const int f_prev2 = (f_prev == 0) ? F_SLOTS - 1 : f_prev - 1;  // row r-2 (= r+1)
    const int g_next = (g_cur + 1) & (G_SLOTS - 1);
    const int g_prev2 = (g_cur + 2) & (G_SLOTS - 1);  // row r-2
    issue_row(k + 1, f_next, g_next);
    cp_async_wait_1();  // this thread's copies of row k have landed

    // ===================== phase A: row r =====================
    const bool row_ok = pery || (r >= 0 && r < ny);
    const int rn = pery ? wrap_index(r, ny) : r;
    NodeState<Real> ns;
    ns.rho = Real(1); ns.inv_rho = Real(1); ns.drho = Real(0); ns.ux = Real(0); ns.uy = Real(0);
    ns.T = T0; ns.dT = Real(0); ns.coef = Real(0); ns.dpsi = Real(0);
    if (col_ok && row_ok) {
      Real* fs = sF + f_cur * 9 * NS + s;
      Real* gs = sG + g_cur * 9 * NS + s;
      Real fc[9], gc[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        fc[i] = fs[i * NS];
        gc[i] = THERMAL ? gs[i * NS] : Real(0);
      }
      const NodeBC nb{!pery && rn == 0, !pery && !pool && rn == ny - 1, inl, outl, pool && rn == ny - 1};
      if (!local && (nb.wlo || nb.whi || inl || outl || nb.top)) {
        boundary_fill<Real, THERMAL>(fc, gc, nb, I, sC, Gin, plane, pitch, rn * pitch + xn, xn, perx, step);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          fs[i * NS] = fc[i];
          if (THERMAL) gs[i * NS] = gc[i];
        }
      }
      ns = node_state<Real, THERMAL>(fc, gc, sC, multiphase, hazi);
      if (ns.bad) atomicOr(&st->status, STATUS_UNSTABLE);
      sPsi[f_cur * NS + s] = ns.dpsi;
      const bool out_row = r >= tile.y0 && r < tile.y1;
      if (post_open && !local && (inl || outl) && out_col && out_row) {
        // mass this node's pull took in minus the mass the pull let out of the lattice: in, the
        // open-end links that boundary_fill set; out, this node's post-collision populations
        // that point out of the open end (no node pulls them; at a wall row the diagonal one is
        // bounced back instead).  Summed over the open ends this is the change of the total
        // mass from the previous step to this one, up to the rounding of the collision.
        const bool lo = rn == 0, hi = rn == ny - 1;
        const int node = rn * pitch + xn;
        auto fload = [&](int i) {
          const int k = i * plane + node;
          return idx_ok(I.st, k, 9LL * plane) ? (double)ld_ro(Fin + k) : 0.0;
        };
        if (inl)
          acc_open += (double)fc[1] + (lo ? 0.0 : (double)fc[5]) + (hi ? 0.0 : (double)fc[8]) -
                      (fload(3) + (hi ? 0.0 : fload(6)) + (lo ? 0.0 : fload(7)));
        else
          acc_open += (double)fc[3] + (lo ? 0.0 : (double)fc[6]) + (hi ? 0.0 : (double)fc[7]) -
                      (fload(1) + (hi ? 0.0 : fload(5)) + (lo ? 0.0 : fload(8)));
      }
      const Real hmc = ns.hmc;
      ns.hmc = Real(0);  // becomes the source term of this node (output nodes of the step only)
      if (hazi && out_col && out_row) {
        // temporal density gradient rho^n - rho^(n-1), both as deviations from rho_ref; this
        // thread owns the node's history (read, then overwritten with rho^n)
        const int kp = rn * pitch + xn;
        if (idx_ok(I.st, kp, I.plane)) {
          Real* rp = rho_prev + kp;
          if (MODE == MODE_STEP) ns.hmc = hmc * (ns.drho - *rp);
          if (MODE == MODE_STEP || MODE == MODE_MOMENTS) *rp = ns.drho;
        }
      }
      if ((MODE == MODE_STEP || MODE == MODE_MOMENTS) && out_col && out_row) {
        acc_m += ns.drho;
        if (THERMAL) {
          acc_e += ns.dT;
          if (!pery && rn == 0 && xn >= I.heater_x0 && xn < I.heater_x0 + I.heater_len) acc_h += ns.dT;
        }
        if (bubbles && ns.drho < sC.drho_vapor) {
          acc_va += 1.0f;
          if (zone_col) acc_zv += 1.0f;
          if (!pery && rn == 0) {
            acc_wv += 1.0f;
            if (xn >= I.heater_x0 && xn < I.heater_x0 + I.heater_len) acc_hv += 1.0f;
          }
        }
        if (MODE == MODE_STEP && channel && rn == ny / 2 && (xn == 1 || xn == nx - 2)) {
          if (xn == 1) st->p_probe[2 * (step & 1)] = (double)ns.p;
          if (xn == nx - 2) st->p_probe[2 * (step & 1) + 1] = (double)ns.p;
          __threadfence();
        }
      }
      if (MODE == MODE_POPS && out_col && out_row) {
        const int oo = rn * pitch + xn;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          if (!idx_ok(I.st, i * plane + oo, 9LL * plane)) continue;
          Fout[i * plane + oo] = fc[i];
          if (THERMAL) Gout[i * plane + oo] = gc[i];
        }
      }
    }
    if (MODE == MODE_POPS || MODE == MODE_MOMENTS) {
      f_cur = f_next;
      g_cur = g_next;
      continue;
    }
    __syncthreads();

    // ===================== phase B: row q = r - 1 =====================
    const int q = r - 1;
    // STEP needs u_act from row y0 - 1 (divergence at y0); FIELDS only on its output rows
    const int qmin = (MODE == MODE_STEP) ? tile.y0 - 1 : tile.y0;
    if (q >= qmin && f_col && (pery || (q >= 0 && q < ny))) {
      const bool sol_m = !pery && q == 0;                // row q-1 is the bottom wall
      const bool sol_p = !pery && !pool && q == ny - 1;  // row q+1 is the top wall
      Real Fx = Real(0), Fy = Real(0);
      if (multiphase) {
        const Real* P0 = sPsi + f_prev * NS;
        // above the pool's top row: the zero-gradient ghost row repeats row q
        const Real* Pp = (pool && q == ny - 1) ? P0 : sPsi + f_cur * NS;
        const Real* Pm = sPsi + f_prev2 * NS;
        sc_force<Real>(P0[s], P0[sp], P0[sm], sol_p ? Real(0) : Pp[s], sol_p ? Real(0) : Pp[sp],
                       sol_p ? Real(0) : Pp[sm], sol_m ? Real(0) : Pm[s], sol_m ? Real(0) : Pm[sp],
                       sol_m ? Real(0) : Pm[sm], sol_m, sol_p, sC, Fx, Fy);
      }
      Fy -= (drho_p + sRra) * sC.g_a;  // Eq. 14, gravity along -y
      // FP64 reuses phase A's reciprocal (several FP64 instructions); FP32
      // recomputes its cheap approximate one rather than hold another register
      const Real inv_rho = sizeof(Real) == 8 ? inv_rho_p : fast_rcp(rho_p);
      const Real dux = Fx * inv_rho, duy = Fy * inv_rho;
      const Real uax = ux_p + Real(0.5) * dux, uay = uy_p + Real(0.5) * duy;  // Eq. 7
      sUx[f_prev * NS + s] = uax;
      sUy[f_prev * NS + s] = uay;
      const bool out_q = out_col && q >= tile.y0 && q < tile.y1;
      if (MODE == MODE_STEP && out_q) {
        collide_f<Real>(StridedPops<Real>{sF + f_prev * 9 * NS + s, NS}, plane_out(Fout, q * pitch + xn, plane, I.st, 9LL * plane),
                        rho_p, drho_p, ux_p, uy_p, dux, duy, sC.omega_f);
        if (channel && xn == 0) acc_fi += rho_p * uax;
        if (channel && xn == nx - 1) acc_fo += rho_p * uax;
      }
      if (MODE == MODE_FIELDS && out_q) {
        double* out = static_cast<double*>(I.f[(step + 1) & 1]);
        const long long n = (long long)nx * ny;
        const long long oo = (long long)q * nx + xn;
        if (idx_ok(I.st, oo, n) && idx_ok(I.st, 3 * n + oo, 9LL * plane * (long long)sizeof(Real) / 8)) {
          out[oo] = (double)rho_p;
          out[n + oo] = (double)uax;
          out[2 * n + oo] = (double)uay;
          out[3 * n + oo] = (double)T_p;
        }
      }
    }
    __syncthreads();

    // ===================== phase C: row q2 = r - 2 =====================
    if (THERMAL && MODE == MODE_STEP) {
      const int q2 = r - 2;
      if (out_col && q2 >= tile.y0 && q2 < tile.y1) {
        // second-order central differences of u_act (ghost copy at open ends); on a row next
        // to a wall the wall-normal derivative is the one-sided difference over the fluid rows
        const Real uxE = sUx[f_prev2 * NS + sp], uxW = sUx[f_prev2 * NS + sm];
        Real uyN = sUy[f_prev * NS + s];
        if (pool && q2 == ny - 1) uyN = sUy[f_prev2 * NS + s];  // pool top: the ghost row repeats row q2
        const Real uyS = sUy[f_cur * NS + s];  // slot of row r-3
        const bool wall_lo = !pery && q2 == 0, wall_hi = !pery && !pool && q2 == ny - 1;
        Real dyu = Real(0.5) * (uyN - uyS);
        if (wall_lo || wall_hi) {
          const Real uyC = sUy[f_prev2 * NS + s];
          dyu = (wall_lo && wall_hi) ? Real(0) : (wall_lo ? uyN - uyC : uyC - uyS);
        }
        const Real divu = Real(0.5) * (uxE - uxW) + dyu;
        Real phi = coef_p2 * divu;
        if (hazi) phi += hm_p2;
        collide_g<Real>(StridedPops<Real>{sG + g_prev2 * 9 * NS + s, NS}, plane_out(Gout, q2 * pitch + xn, plane, I.st, 9LL * plane),
                        T_p2, dT_p2, sUx[f_prev2 * NS + s], sUy[f_prev2 * NS + s], phi, sC.omega_g);
      }
    }

    T_p2 = T_p;
    dT_p2 = dT_p;
    coef_p2 = coef_p;
    if (hazi) {
      hm_p2 = hm_p;
      hm_p = ns.hmc;
    }
    rho_p = ns.rho;
    inv_rho_p = ns.inv_rho;
    drho_p = ns.drho;
    ux_p = ns.ux;
    uy_p = ns.uy;
    T_p = ns.T;
    dT_p = ns.dT;
    coef_p = ns.coef;
    f_cur = f_next;
    g_cur = g_next;
  }

  if (MODE != MODE_STEP && MODE != MODE_MOMENTS) return;

  // ---------------- per-tile partials into the launch's totals ----------------
  double acc[NPART] = {(double)acc_m,  (double)acc_e,  (double)acc_h,  (double)acc_fi, (double)acc_fo,
                       (double)acc_va, (double)acc_wv, (double)acc_hv, (double)acc_zv};
  post_partials<BLOCK, THERMAL, MODE>(I, st, tile, acc, sRed, &sLast, step, post_open, acc_open);
}

// Resident CTAs per SM the step kernels are compiled for (register budget).  The FP32 kernel
// with the interior path is compiled for 4 CTAs of 128 threads per SM (up to 128 registers):
// measured faster than 5 at 96 registers or 6 at 80, both of which also leave less L1 beside
// the shared-memory rings.
template <typename Real, int B, bool INTERIOR>
constexpr int step_min_blocks() {
  return sizeof(Real) == 4 ? (B <= 64 ? 10 : (B <= 128 ? (INTERIOR ? 4 : 5) : 2)) : (B <= 64 ? 4 : (B <= 128 ? 2 : 1));
}

template <typename Real, bool THERMAL, int B, int MODE, bool FULL = true, bool PCONST = false, bool INTERIOR = false>
__global__ void __launch_bounds__(B, (step_min_blocks<Real, B, INTERIOR>()))
lbm_fused_kernel(const Inst* __restrict__ insts, const Tile* __restrict__ tiles,
                 const __grid_constant__ KParams<Real> kp) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  __shared__ StepShared<Real, B, PCONST> sh;
  fused_tile<Real, THERMAL, B, MODE, FULL, PCONST, INTERIOR>(insts, tiles[blockIdx.x], kp, dyn_smem, sh);
}

// ---------------------------------------------------------------------------
// Persistent form of the step: one cooperative launch advances the instances nsteps steps.
// Every CTA draws tiles from a per-step counter and runs them with the same tile body as
// lbm_fused_kernel; the tile that completes a step still finishes it (totals, record, mean
// density for the next step's buoyancy), and a grid-wide barrier separates the steps.  The
// launch is cooperative, so every CTA is resident and the barrier cannot wait on a CTA that
// has not started; each wait is still bounded (BARRIER_WAIT_NS of polling, or max_polls
// polls), after which the CTA marks the barrier, sets STATUS_TIMEOUT on its instance and
// returns, and the others stop at their next poll.  Between steps no launch is needed, which
// takes the launch gap and the kernel boundary off lattices whose step is a single wave.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier: false if this CTA gave up waiting (or another one did).
__device__ __forceinline__ bool grid_barrier(GridBar* bar, unsigned nblocks, unsigned max_polls, int* s_ok) {
  __syncthreads();  // the CTA's work of this step is done
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &bar->gen;
    volatile unsigned* vstatus = &bar->status;
    const unsigned gen = *vgen;  // read before arriving: it cannot advance before this CTA arrives
    __threadfence();             // this CTA's writes are visible before its arrival
    int ok = 1;
    if (atomicAdd(&bar->count, 1u) == nblocks - 1) {
      atomicExch(&bar->count, 0u);  // nobody touches count again before gen advances
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const unsigned long long t0 = global_ns();
      unsigned polls = 0;
      while (*vgen == gen) {
        ++polls;
        if ((max_polls != 0 && polls >= max_polls) || *vstatus != 0 || global_ns() - t0 > BARRIER_WAIT_NS) {
          ok = *vgen != gen;  // released at the last moment
          break;
        }
      }
    }
    if (!ok) atomicOr(&bar->status, 1u);
    __threadfence();  // the other CTAs' writes of this step are visible after the barrier
    *s_ok = ok && *vstatus == 0;  // a CTA that gave up ends the launch for all
  }
  __syncthreads();
  return *s_ok != 0;
}

// Band of row y in an instance's overlapped tiling (tall bands first, then short ones).
__device__ __forceinline__ int flow_band(const FlowInst& f, int y) {
  const int ytall = f.tall_rows * f.tall_count;
  return y < ytall ? y / f.tall_rows : f.tall_count + (y - ytall) / f.short_rows;
}

// Thread 0 polls *p until it reaches `need`, at most max_polls polls (0: no cap) and
// BARRIER_WAIT_NS from t0, and gives up early once another CTA has given up (bar->status).
template <typename T>
__device__ __forceinline__ bool flow_wait(const volatile T* p, T need, const GridBar* bar, unsigned max_polls,
                                          unsigned& polls, unsigned long long t0) {
  const volatile unsigned* vstatus = &bar->status;
  while (*p < need) {
    ++polls;
    if ((max_polls != 0 && polls >= max_polls) || *vstatus != 0 || global_ns() - t0 > BARRIER_WAIT_NS)
      return *p >= need;
  }
  return true;
}

// The overlapped persistent loop (see FlowPlan): nsteps steps of the launch's tiles in
// (step, tile) ticket order.  The launch's first CTA records every instance's step count
// before a grid barrier, so that the tickets of step k of the launch run step step0 + k of
// their instance.  A ticket's tile waits, on thread 0 with bounded polls, for
//  - the tiles of its instance holding rows y0 - 3 .. y1 + 2 and columns x0 - 3 .. x1 + 2
//    (what its pulls read, wrapped where the lattice is periodic) to have finished the
//    previous step: the tiles it reads from and those that read what it overwrites;
//  - the instance's step two back to be complete (its diagnostics record and mean density);
//  - the instance's open-end tiles of the previous step to have posted the mass through the
//    open ends;
// then runs with the buoyancy mean rho_avg(s - 2) + (mass through the open ends in s - 1) / N,
// which is the previous step's mean up to the rounding of one collision, whatever the timing.
// Tickets are drawn in order and a tile waits only for tickets drawn before it, all of them
// held by resident CTAs, so the loop always progresses; a CTA that gives up marks the launch
// (bar->status), every CTA then stops at its next wait, and the instance reports a timeout.
template <typename Real, bool THERMAL, int B, bool FULL, bool PCONST, bool INTERIOR>
__device__ __forceinline__ void overlapped_steps(const Inst* __restrict__ insts, const Tile* __restrict__ tiles,
                                                 int ntiles, int nsteps, GridBar* bar, unsigned max_polls,
                                                 const KParams<Real>& kp, const FlowPlan& flow,
                                                 unsigned char* dyn_smem, StepShared<Real, B, PCONST>& sh) {
  __shared__ long long s_q;
  __shared__ int s_ok;
  __shared__ double s_rho;
  if (blockIdx.x == 0) {
    for (int i = threadIdx.x; i < flow.ninst; i += B) flow.step0[i] = (PCONST ? kp.I.st : insts[i].st)->step;
  }
  if (!grid_barrier(bar, gridDim.x, max_polls, &s_ok)) {
    if (threadIdx.x == 0) atomicOr(&(PCONST ? kp.I.st : insts[tiles[0].inst].st)->status, STATUS_TIMEOUT);
    return;
  }
  const long long total = (long long)nsteps * ntiles;
  for (;;) {
    if (threadIdx.x == 0) s_q = (long long)atomicAdd(&bar->claim, 1ull);
    __syncthreads();
    const long long q = s_q;
    if (q >= total) return;
    const int k = (int)(q / ntiles);
    const Tile tile = tiles[q - (long long)k * ntiles];
    const Inst& Ii = PCONST ? kp.I : insts[tile.inst];
    const FlowInst& fi = flow.inst ? flow.inst[tile.inst] : flow.single;
    InstState* st = Ii.st;
    const long long step = flow.step0[tile.inst] + k;
    if (threadIdx.x == 0) {
      bool ok = true;
      double rho = 0.0;
      if (k == 0) {
        rho = st->rho_avg[(step - 1) & 1];
      } else {
        unsigned polls = 0;
        const unsigned long long t0 = global_ns();
        const unsigned long long need = (unsigned long long)k;  // steps each neighbour has finished
        const int ny = Ii.ny, nx = Ii.nx;
        const long long ncells = (long long)fi.nbands * fi.strips;
        // the rows and columns this tile's pulls read: its own, 3 rows and 3 columns around
        int ylo = tile.y0 - 3, yhi = tile.y1 + 2;
        if (!fi.pery) {
          ylo = ylo < 0 ? 0 : ylo;
          yhi = yhi > ny - 1 ? ny - 1 : yhi;
        } else if (yhi - ylo + 1 >= ny) {
          ylo = 0;
          yhi = ny - 1;
        }
        const int x1 = tile.x0 + fi.tile_w < nx ? tile.x0 + fi.tile_w : nx;
        int xlo = tile.x0 - 3, xhi = x1 + 2;
        if (!fi.perx) {
          xlo = xlo < 0 ? 0 : xlo;
          xhi = xhi > nx - 1 ? nx - 1 : xhi;
        } else if (xhi - xlo + 1 >= nx) {
          xlo = 0;
          xhi = nx - 1;
        }
        const int ytall = fi.tall_rows * fi.tall_count;
        for (int y = ylo; ok && y <= yhi;) {
          const int yy = y < 0 ? y + ny : (y >= ny ? y - ny : y);
          const int b = flow_band(fi, yy);
          for (int x = xlo; ok && x <= xhi;) {
            const int xx = x < 0 ? x + nx : (x >= nx ? x - nx : x);
            const int j = xx / fi.tile_w;
            const long long cell = (long long)b * fi.strips + j;
            if (idx_ok(st, cell, ncells))
              ok = flow_wait<unsigned long long>(flow.cell_done + fi.cell_base + cell, need, bar, max_polls, polls,
                                                 t0);
            const int xend = (j + 1) * fi.tile_w;
            x += (xend < nx ? xend : nx) - xx;  // first column of the next strip
          }
          const int bend = b < fi.tall_count ? (b + 1) * fi.tall_rows
                                             : ytall + (b - fi.tall_count + 1) * fi.short_rows;
          y += (bend < ny ? bend : ny) - yy;  // first row of the next band
        }
        if (ok) ok = flow_wait<long long>(&st->step, step - 1, bar, max_polls, polls, t0);
        if (ok && fi.n_open > 0)
          ok = flow_wait<unsigned>(&st->open_posted[(step - 1) & 3], (unsigned)fi.n_open, bar, max_polls, polls, t0);
        __threadfence();  // what the awaited tiles wrote is visible after their counts
        if (ok) {
          const long long m = *reinterpret_cast<const volatile long long*>(&st->open_mass[(step - 1) & 3]);
          rho = *reinterpret_cast<const volatile double*>(&st->rho_avg[(step - 2) & 1]) +
                (double)m * Ii.fix_unscale[3] / ((double)Ii.nx * (double)Ii.ny);
        }
      }
      if (!ok) {
        atomicOr(&bar->status, 1u);
        atomicOr(&st->status, STATUS_TIMEOUT);
      }
      s_ok = ok;
      s_rho = rho;
    }
    __syncthreads();
    if (!s_ok) return;
    TileStep ts;
    ts.step = step;
    // a first step reads the populations in place; the flag stays set until that step of the
    // instance completes, which needs this tile
    ts.local = k == 0 && st->local_read != 0;
    ts.post_open = true;
    ts.rho_avg_prev = s_rho;
    fused_tile<Real, THERMAL, B, MODE_STEP, FULL, PCONST, INTERIOR>(insts, tile, kp, dyn_smem, sh, ts);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();  // the tile's populations are written before its count
      const long long cell = (long long)flow_band(fi, tile.y0) * fi.strips + tile.x0 / fi.tile_w;
      if (idx_ok(st, cell, (long long)fi.nbands * fi.strips)) atomicAdd(flow.cell_done + fi.cell_base + cell, 1ull);
    }
  }
}

template <typename Real, bool THERMAL, int B, bool FULL, bool PCONST, bool INTERIOR>
__global__ void __launch_bounds__(B, (step_min_blocks<Real, B, INTERIOR>()))
lbm_persistent_kernel(const Inst* __restrict__ insts, const Tile* __restrict__ tiles, int ntiles, int nsteps,
                      GridBar* bar, unsigned max_polls, const __grid_constant__ KParams<Real> kp,
                      const __grid_constant__ FlowPlan flow) {
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  __shared__ StepShared<Real, B, PCONST> sh;
  __shared__ int s_tile, s_ok;
  int first_inst = -1;
  // With a CTA per tile (one wave) every CTA runs tile blockIdx.x; otherwise the CTAs draw tiles
  // from the step's counter, so that the tall bands dispatched first are shared out as they end.
  const bool one_wave = ntiles <= (int)gridDim.x;
  if (!one_wave && flow.enabled) {
    overlapped_steps<Real, THERMAL, B, FULL, PCONST, INTERIOR>(insts, tiles, ntiles, nsteps, bar, max_polls, kp,
                                                               flow, dyn_smem, sh);
    return;
  }
  for (int n = 0; n < nsteps; ++n) {
    if (one_wave) {
      const Tile tile = tiles[blockIdx.x];
      first_inst = tile.inst;
      fused_tile<Real, THERMAL, B, MODE_STEP, FULL, PCONST, INTERIOR>(insts, tile, kp, dyn_smem, sh);
    } else {
      if (blockIdx.x == 0 && threadIdx.x == 0) bar->next[(n + 1) & 1] = 0u;  // last drawn from in step n - 1
      for (;;) {
        if (threadIdx.x == 0) s_tile = (int)atomicAdd(&bar->next[n & 1], 1u);
        __syncthreads();
        const int t = s_tile;
        __syncthreads();
        if (t >= ntiles) break;
        const Tile tile = tiles[t];
        if (first_inst < 0) first_inst = tile.inst;
        fused_tile<Real, THERMAL, B, MODE_STEP, FULL, PCONST, INTERIOR>(insts, tile, kp, dyn_smem, sh);
        __syncthreads();
      }
    }
    if (n + 1 < nsteps && !grid_barrier(bar, gridDim.x, max_polls, &s_ok)) {
      if (threadIdx.x == 0 && first_inst >= 0) atomicOr(&insts[first_inst].st->status, STATUS_TIMEOUT);
      if (threadIdx.x == 0 && PCONST) atomicOr(&kp.I.st->status, STATUS_TIMEOUT);
      return;
    }
  }
}

template <typename Real, bool THERMAL, int B, bool FULL, bool PCONST, bool INTERIOR>
cudaError_t launch_persistent_one(const Inst* d_inst, const Tile* d_tiles, int ntiles, int nsteps, GridBar* bar,
                                  unsigned max_polls, cudaStream_t s, const KParams<Real>& kp,
                                  const FlowPlan& flow) {
  constexpr size_t smem = step_smem_bytes<Real, THERMAL, B, INTERIOR>();
  auto fn = lbm_persistent_kernel<Real, THERMAL, B, FULL, PCONST, INTERIOR>;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, B, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int grid = ntiles < sms * per_sm ? ntiles : sms * per_sm;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(B);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, d_inst, d_tiles, ntiles, nsteps, bar, max_polls, kp, flow);
}

template <typename Real, bool THERMAL, int B, bool FULL, bool PCONST, bool INTERIOR>
int persistent_resident() {
  constexpr size_t smem = step_smem_bytes<Real, THERMAL, B, INTERIOR>();
  auto fn = lbm_persistent_kernel<Real, THERMAL, B, FULL, PCONST, INTERIOR>;
  int n = 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, B, smem) != cudaSuccess)
    return 0;
  return n;
}

// Persistent launch for one precision: the lean form with the interior path (single instance:
// constants as the kernel parameter), or the full form.
template <typename Real, bool THERMAL, int B>
cudaError_t launch_persistent_cols(bool full, bool interior, const Inst* d_inst, const Tile* d_tiles, int ntiles,
                                   int nsteps, GridBar* bar, unsigned max_polls, cudaStream_t s, const Inst* h_inst,
                                   const FlowPlan& flow) {
  KParams<Real> kp{};
  if (full) return launch_persistent_one<Real, THERMAL, B, true, false, false>(d_inst, d_tiles, ntiles, nsteps, bar,
                                                                               max_polls, s, kp, flow);
  if (h_inst) {
    kp.I = *h_inst;
    fill_consts<Real>(kp.C, *h_inst, h_inst->rho_ref);
    if (interior)
      return launch_persistent_one<Real, THERMAL, B, false, true, true>(d_inst, d_tiles, ntiles, nsteps, bar,
                                                                        max_polls, s, kp, flow);
    return launch_persistent_one<Real, THERMAL, B, false, true, false>(d_inst, d_tiles, ntiles, nsteps, bar,
                                                                       max_polls, s, kp, flow);
  }
  if (interior)
    return launch_persistent_one<Real, THERMAL, B, false, false, true>(d_inst, d_tiles, ntiles, nsteps, bar,
                                                                       max_polls, s, kp, flow);
  return launch_persistent_one<Real, THERMAL, B, false, false, false>(d_inst, d_tiles, ntiles, nsteps, bar, max_polls,
                                                                      s, kp, flow);
}

template <typename Real, bool THERMAL, int B>
int persistent_resident_cols(bool full, bool interior, bool single) {
  if (full) return persistent_resident<Real, THERMAL, B, true, false, false>();
  if (single) return interior ? persistent_resident<Real, THERMAL, B, false, true, true>()
                              : persistent_resident<Real, THERMAL, B, false, true, false>();
  return interior ? persistent_resident<Real, THERMAL, B, false, false, true>()
                  : persistent_resident<Real, THERMAL, B, false, false, false>();
}

template <typename Real>
cudaError_t launch_persistent_precision(int thermal, int cols, bool full, bool interior, const Inst* d_inst,
                                        const Tile* d_tiles, int ntiles, int nsteps, GridBar* bar, unsigned max_polls,
                                        cudaStream_t s, const Inst* h_inst, const FlowPlan& flow) {
  if (ntiles <= 0 || nsteps <= 0) return cudaSuccess;
#define PPLBM_PERSIST(TH, COLS) \
  launch_persistent_cols<Real, TH, COLS>(full, interior, d_inst, d_tiles, ntiles, nsteps, bar, max_polls, s, h_inst, flow)
  if (thermal) {
    switch (cols) {
      case 64: return PPLBM_PERSIST(true, 64);
      case 128: return PPLBM_PERSIST(true, 128);
      case 256: return PPLBM_PERSIST(true, 256);
    }
  } else {
    switch (cols) {
      case 64: return PPLBM_PERSIST(false, 64);
      case 128: return PPLBM_PERSIST(false, 128);
      case 256: return PPLBM_PERSIST(false, 256);
    }
  }
#undef PPLBM_PERSIST
  return cudaErrorInvalidValue;
}

template <typename Real>
int persistent_resident_precision(int thermal, int cols, bool full, bool interior, bool single) {
  if (thermal) {
    switch (cols) {
      case 64: return persistent_resident_cols<Real, true, 64>(full, interior, single);
      case 128: return persistent_resident_cols<Real, true, 128>(full, interior, single);
      case 256: return persistent_resident_cols<Real, true, 256>(full, interior, single);
    }
  } else {
    switch (cols) {
      case 64: return persistent_resident_cols<Real, false, 64>(full, interior, single);
      case 128: return persistent_resident_cols<Real, false, 128>(full, interior, single);
      case 256: return persistent_resident_cols<Real, false, 256>(full, interior, single);
    }
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Initialisation: f = f^eq(rho, u) (Eq. 3), g = g^eq(T, u) (Eq. 18) into buffer 0,
// stored in the library's storage form (deviations in FP32).
// ---------------------------------------------------------------------------
template <typename Real>
__device__ __forceinline__ void write_equilibrium(const Inst& I, long long node, double rho, double ux,
                                                  double uy, double T) {
  // The reference parts are taken off in FP64; the rest is computed in the storage
  // precision (FP32 storage keeps FP32 rounding of the deviations either way, and FP64
  // arithmetic is scarce on this GPU).
  if (!idx_ok(I.st, node, I.plane)) return;  // node of plane 0: every plane's element is then in its buffer
  Real* F = static_cast<Real*>(I.f[0]);
  Real* Gb = static_cast<Real*>(I.g[0]);
  const Real drho = Real(rho - I.rho_ref), dT = Real(T - I.T_ref);
  static_cast<Real*>(I.rho_prev)[node] = drho;  // no density change before the first step
  const Real r = Real(rho), t = Real(T), vx = Real(ux), vy = Real(uy);
  const Real usq = vx * vx + vy * vy;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const Real cu = Real(lat_cx(i)) * vx + Real(lat_cy(i)) * vy;
    const Real w = lat_w<Real>(i);
    const Real poly = Real(3) * cu + Real(4.5) * cu * cu - Real(1.5) * usq;
    F[i * I.plane + node] = w * (drho + r * poly);
    Gb[i * I.plane + node] = w * (dT + t * poly);
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
template <typename Real, bool THERMAL, int B, int MODE, bool FULL, bool PCONST = false, bool INTERIOR = false>
cudaError_t launch_one(const Inst* d_inst, const Tile* d_tiles, int ntiles, cudaStream_t s,
                       const KParams<Real>& kp = KParams<Real>{}) {
  constexpr size_t smem = step_smem_bytes<Real, THERMAL, B, INTERIOR>();
  // the dynamic shared-memory opt-in is per device; remember which devices have it
  static unsigned long long configured = 0ull;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(configured & bit)) {
    e = cudaFuncSetAttribute(lbm_fused_kernel<Real, THERMAL, B, MODE, FULL, PCONST, INTERIOR>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured |= bit;
  }
  lbm_fused_kernel<Real, THERMAL, B, MODE, FULL, PCONST, INTERIOR><<<ntiles, B, smem, s>>>(d_inst, d_tiles, kp);
  return cudaGetLastError();
}

// Step-kernel CTAs resident per SM on the current device (at least 1).
template <typename Real, bool THERMAL, int B, bool INTERIOR>
int resident_one() {
  constexpr size_t smem = step_smem_bytes<Real, THERMAL, B, INTERIOR>();
  auto fn = lbm_fused_kernel<Real, THERMAL, B, MODE_STEP, false, INTERIOR, INTERIOR>;
  int n = 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, B, smem) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

template <typename Real, bool INTERIOR>
int resident_form(int thermal, int cols) {
  if (thermal) {
    switch (cols) {
      case 64: return resident_one<Real, true, 64, INTERIOR>();
      case 128: return resident_one<Real, true, 128, INTERIOR>();
      case 256: return resident_one<Real, true, 256, INTERIOR>();
    }
  } else {
    switch (cols) {
      case 64: return resident_one<Real, false, 64, INTERIOR>();
      case 128: return resident_one<Real, false, 128, INTERIOR>();
      case 256: return resident_one<Real, false, 256, INTERIOR>();
    }
  }
  return 1;
}

template <typename Real>
int resident_precision(int thermal, int cols, bool interior) {
  return interior ? resident_form<Real, true>(thermal, cols) : resident_form<Real, false>(thermal, cols);
}

// h_inst: the host copy of the launch's only instance (its constants then travel as a kernel
// parameter to the lean step), or null for launches over several instances.
template <typename Real, bool THERMAL, int B>
cudaError_t launch_cols(int mode, bool full, bool interior, const Inst* d_inst, const Tile* d_tiles, int ntiles,
                        cudaStream_t s, const Inst* h_inst) {
  switch (mode) {
    case MODE_STEP:
      if (full) return launch_one<Real, THERMAL, B, MODE_STEP, true>(d_inst, d_tiles, ntiles, s);
      if (h_inst) {
        KParams<Real> kp;
        kp.I = *h_inst;
        fill_consts<Real>(kp.C, *h_inst, h_inst->rho_ref);
        if (interior) return launch_one<Real, THERMAL, B, MODE_STEP, false, true, true>(d_inst, d_tiles, ntiles, s, kp);
        return launch_one<Real, THERMAL, B, MODE_STEP, false, true>(d_inst, d_tiles, ntiles, s, kp);
      }
      if (interior) return launch_one<Real, THERMAL, B, MODE_STEP, false, false, true>(d_inst, d_tiles, ntiles, s);
      return launch_one<Real, THERMAL, B, MODE_STEP, false>(d_inst, d_tiles, ntiles, s);
    case MODE_FIELDS: return launch_one<Real, THERMAL, B, MODE_FIELDS, true>(d_inst, d_tiles, ntiles, s);
    case MODE_POPS: return launch_one<Real, THERMAL, B, MODE_POPS, true>(d_inst, d_tiles, ntiles, s);
    case MODE_MOMENTS: return launch_one<Real, THERMAL, B, MODE_MOMENTS, true>(d_inst, d_tiles, ntiles, s);
  }
  return cudaErrorInvalidValue;
}

// interior: the step takes the kernel with its interior path (LBM_KERNEL_INTERIOR).
template <typename Real>
cudaError_t launch_precision(int thermal, int cols, int mode, bool full, bool interior, const Inst* d_inst,
                             const Tile* d_tiles, int ntiles, cudaStream_t s, const Inst* h_inst) {
  if (ntiles <= 0) return cudaSuccess;
  if (thermal) {
    switch (cols) {
      case 64: return launch_cols<Real, true, 64>(mode, full, interior, d_inst, d_tiles, ntiles, s, h_inst);
      case 128: return launch_cols<Real, true, 128>(mode, full, interior, d_inst, d_tiles, ntiles, s, h_inst);
      case 256: return launch_cols<Real, true, 256>(mode, full, interior, d_inst, d_tiles, ntiles, s, h_inst);
    }
  } else {
    switch (cols) {
      case 64: return launch_cols<Real, false, 64>(mode, full, interior, d_inst, d_tiles, ntiles, s, h_inst);
      case 128: return launch_cols<Real, false, 128>(mode, full, interior, d_inst, d_tiles, ntiles, s, h_inst);
      case 256: return launch_cols<Real, false, 256>(mode, full, interior, d_inst, d_tiles, ntiles, s, h_inst);
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
