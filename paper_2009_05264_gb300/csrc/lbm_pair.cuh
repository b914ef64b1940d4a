// FP32 fused step with two adjacent columns per thread and packed FP32 arithmetic.
//
// Same time step as lbm_fused_kernel (Sec. 2 of Mukherjee, Basu & Mondal, arXiv
// 2009.05264, with the boundary conditions of Sec. 2.C), organised for the packed
// FP32 instructions of sm_100-class GPUs (FADD2 / FMUL2 / FFMA2 on a register
// pair): thread t updates the nodes x = x0 - 2 + 2t and x + 1, so every
// arithmetic instruction of the moments, equation of state, force and both
// collisions serves two nodes, and the address, index and predicate work of the
// pulls, stores and rings is shared by two nodes.  Populations leave as 8-byte
// stores (x is even and the row pitch a multiple of 32 elements).
//
// Layout requirement: even row pitch and plane size and 8-byte aligned population
// buffers (the library's own layout: pitch a multiple of 32, 256-byte aligned
// buffers).  Callers with other layouts use the scalar kernel.
//
// Tile geometry is that of the scalar kernel with 2B columns: a CTA of B threads
// writes the 2B - 8 output columns [x0, x0 + 2B - 8) and computes two halo columns
// on each side; the last two threads only idle.  Each thread stages the
// populations its two nodes pull in its own shared-memory ring slots (cp.async, one
// row ahead), so, as in the scalar kernel, no thread reads another thread's staged
// data and two barriers per row suffice.
#pragma once

#include "lbm_kernels.cuh"

namespace pplbm {

// ---------------------------------------------------------------------------
// Packed FP32 helpers (two lanes: lane x = node x, lane y = node x + 1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_bc(float c) { return make_float2(c, c); }
__device__ __forceinline__ float2 p_rcp(float2 a) { return make_float2(fast_rcp(a.x), fast_rcp(a.y)); }

// Moments, equation of state and psi of two nodes: the FP32 branch of node_state
// (Eqs. 4, 6, 11, 12, 17; psi as psi - psi_ref from the exact difference forms).
struct PairState {
  float2 rho, drho, ux, uy, T, dT, coef, dpsi, p;
  bool bad0, bad1;
};

template <bool THERMAL>
__device__ __forceinline__ PairState pair_state(const float2 (&fc)[9], const float2 (&gc)[9],
                                                const KConst<float>& C, bool multiphase) {
  PairState o;
  o.drho = p_add(p_add(p_add(fc[0], fc[1]), p_add(fc[2], fc[3])),
                 p_add(p_add(p_add(fc[4], fc[5]), p_add(fc[6], fc[7])), fc[8]));
  o.rho = p_add(p_bc(C.rho_ref), o.drho);
  const float2 jx = p_add(p_add(p_sub(fc[1], fc[3]), p_sub(fc[5], fc[6])), p_sub(fc[8], fc[7]));
  const float2 jy = p_sub(p_add(p_sub(fc[2], fc[4]), p_add(fc[5], fc[6])), p_add(fc[7], fc[8]));
  const float2 inv_rho = p_rcp(o.rho);
  o.ux = p_mul(jx, inv_rho);
  o.uy = p_mul(jy, inv_rho);
  if (THERMAL) {
    o.dT = p_add(p_add(p_add(gc[0], gc[1]), p_add(gc[2], gc[3])),
                 p_add(p_add(p_add(gc[4], gc[5]), p_add(gc[6], gc[7])), gc[8]));
    o.T = p_add(p_bc(C.T_ref), o.dT);
  } else {
    o.dT = p_bc(0.0f);
    o.T = p_bc(C.T0);
  }
  o.dpsi = p_bc(0.0f);
  o.p = p_mul(o.rho, p_bc(1.0f / 3.0f));
  o.coef = p_bc(0.0f);
  float2 dpdT = p_bc(0.0f);
  bool bad0 = !(o.rho.x > 0.0f), bad1 = !(o.rho.y > 0.0f);
  if (multiphase) {
    const float2 rho_c = o.rho, drho_c = o.drho, T_c = o.T, dT_c = o.dT;
    const float2 br = p_mul(p_bc(C.b), rho_c);
    const float2 inv1 = p_rcp(p_sub(p_bc(1.0f), br));
    const float2 invD = p_rcp(p_fma(br, p_sub(p_bc(2.0f), br), p_bc(1.0f)));
    const float2 rr_den = p_mul(p_mul(rho_c, rho_c), invD);
    float2 alpha, sa = p_bc(0.0f), inv_sT = p_bc(0.0f), sT = p_bc(0.0f);
    if (THERMAL) {
      inv_sT = make_float2(fast_rsqrt(T_c.x), fast_rsqrt(T_c.y));
      sT = p_mul(T_c, inv_sT);
      sa = p_fma(p_bc(C.kappa), p_sub(p_bc(1.0f), p_mul(sT, p_bc(C.inv_sqrtTc))), p_bc(1.0f));
      alpha = p_mul(sa, sa);
    } else {
      alpha = p_bc(C.alpha0);
    }
    const float2 rr = p_bc(C.rho_ref);
    // dA = R (drho T inv1 + rr dT) inv_u1r
    float2 dA = p_mul(p_mul(drho_c, T_c), inv1);
    if (THERMAL) dA = p_fma(rr, dT_c, dA);
    dA = p_mul(dA, p_bc(C.R * C.inv_u1r));
    // dB = a alpha drho (rho + rr + 2 b rho rr) / (D D_r)
    const float2 s3 = p_fma(p_bc(2.0f * C.b * C.rho_ref), rho_c, p_add(rho_c, rr));
    float2 dB = p_mul(p_mul(p_mul(p_bc(C.a), alpha), drho_c), p_mul(p_mul(s3, invD), p_bc(C.inv_Dr)));
    if (THERMAL) {
      const float2 dsa = p_mul(p_mul(p_bc(-C.kappa * C.inv_sqrtTc), dT_c), p_rcp(p_add(sT, p_bc(C.sqrtT_r))));
      dB = p_fma(p_mul(p_bc(C.a), dsa), p_mul(p_add(sa, p_bc(C.sa_r)), p_bc(C.rr2_Dr)), dB);
    }
    const float2 dp = p_sub(dA, dB);
    const float2 drad = p_mul(p_fma(drho_c, p_bc(-1.0f / 3.0f), dp), p_bc(C.psi_scale));
    const float2 rad = p_add(p_bc(C.rad_ref), drad);
    const float2 psi = make_float2(fast_sqrt(fmaxf(rad.x, 0.0f)), fast_sqrt(fmaxf(rad.y, 0.0f)));
    const float2 den = p_add(psi, p_bc(C.psi_ref));
    const float2 q = p_mul(drad, p_rcp(den));
    o.dpsi = make_float2(den.x > 0.0f ? q.x : 0.0f, den.y > 0.0f ? q.y : 0.0f);
    o.p = p_add(p_bc(C.p_ref), dp);
    bad0 = bad0 || !(br.x < 1.0f) || !(rad.x >= 0.0f);
    bad1 = bad1 || !(br.y < 1.0f) || !(rad.y >= 0.0f);
    if (THERMAL) {
      const float2 dalpha = p_mul(p_mul(p_bc(-C.kappa * C.inv_sqrtTc), sa), inv_sT);
      dpdT = p_sub(p_mul(p_mul(rho_c, p_bc(C.R)), inv1), p_mul(p_mul(p_bc(C.a), dalpha), rr_den));
    }
  }
  if (THERMAL) {
    bad0 = bad0 || !isfinite(o.T.x);
    bad1 = bad1 || !isfinite(o.T.y);
    o.coef = p_mul(o.T, p_sub(p_bc(1.0f), p_mul(p_mul(dpdT, inv_rho), p_bc(C.inv_cv))));
  }
  o.bad0 = bad0;
  o.bad1 = bad1;
  return o;
}

// Interaction force of Eqs. 9, 10, 14, 15 for two nodes (as sc_force).
__device__ __forceinline__ void pair_force(float2 dc, float2 dE, float2 dW, float2 dN, float2 dNE, float2 dNW,
                                           float2 dS, float2 dSE, float2 dSW, bool sol_m, bool sol_p,
                                           const KConst<float>& C, float2& Fx, float2& Fy) {
  const float2 G2 = p_bc(C.G2), Gh = p_bc(C.Gh);
  const float2 t1x = p_fma(G2, p_sub(dE, dW), p_mul(Gh, p_add(p_sub(dNE, dNW), p_sub(dSE, dSW))));
  const float2 t1y = p_fma(G2, p_sub(dN, dS), p_mul(Gh, p_sub(p_add(dNE, dNW), p_add(dSE, dSW))));
  const float2 t2x = p_fma(p_mul(G2, p_sub(dE, dW)), p_add(dE, dW),
                           p_mul(Gh, p_fma(p_sub(dNE, dNW), p_add(dNE, dNW), p_mul(p_sub(dSE, dSW), p_add(dSE, dSW)))));
  const float2 t2y = p_fma(p_mul(G2, p_sub(dN, dS)), p_add(dN, dS),
                           p_mul(Gh, p_fma(p_sub(dNE, dSE), p_add(dNE, dSE), p_mul(p_sub(dNW, dSW), p_add(dNW, dSW)))));
  const float2 lead = p_fma(p_bc(C.beta), dc, p_bc(C.psi_ref));
  const float2 nmix = p_bc(-C.mix);
  Fx = p_fma(nmix, t2x, p_mul(p_sub(p_bc(0.0f), lead), t1x));
  Fy = p_fma(nmix, t2y, p_mul(p_sub(p_bc(0.0f), lead), t1y));
  if (sol_m) Fy = p_add(Fy, p_fma(dc, p_bc(C.wall1), p_bc(C.wall0)));
  if (sol_p) Fy = p_sub(Fy, p_fma(dc, p_bc(C.wall1), p_bc(C.wall0)));
}

// Store one plane's pair of populations: 8 bytes when both nodes are in the domain.
__device__ __forceinline__ void pair_store(float* p, float2 v, bool both) {
  if (both)
    *reinterpret_cast<float2*>(p) = v;
  else
    p[0] = v.x;
}

// BGK + exact-difference collision of f (Eqs. 2, 3, 5) for two nodes, pairwise over
// opposite directions as in collide_f.
__device__ __forceinline__ void pair_collide_f(const float2 (&fs)[9], float* __restrict__ fo, int plane, bool both,
                                               float2 rho, float2 drho, float2 ux, float2 uy, float2 dux, float2 duy,
                                               float omega) {
  const float2 om = p_bc(omega);
  const float2 sx = p_fma(p_bc(2.0f), ux, dux), sy = p_fma(p_bc(2.0f), uy, duy);
  const float2 usq = p_fma(ux, ux, p_mul(uy, uy));
  const float2 r15 = p_mul(p_bc(1.5f), rho);
  // K = omega (drho - 1.5 rho u.u) - 1.5 rho du.(2u + du)
  const float2 K = p_sub(p_mul(om, p_sub(drho, p_mul(r15, usq))), p_mul(r15, p_fma(dux, sx, p_mul(duy, sy))));
  const float2 r45 = p_mul(p_bc(4.5f), rho), r3 = p_mul(p_bc(3.0f), rho), keep = p_bc(1.0f - omega);
  auto pair = [&](int i, int j, float2 cu, float2 cd, float2 cs, float w) {
    const float2 wv = p_bc(w);
    const float2 sym = p_mul(wv, p_fma(r45, p_fma(p_mul(om, cu), cu, p_mul(cd, cs)), K));
    const float2 anti = p_mul(p_mul(wv, r3), p_fma(om, cu, cd));
    const float2 base = p_fma(keep, fs[i], sym);
    const float2 basej = p_fma(keep, fs[j], sym);
    pair_store(fo + i * plane, p_add(base, anti), both);
    pair_store(fo + j * plane, p_sub(basej, anti), both);
  };
  pair_store(fo, p_fma(keep, fs[0], p_mul(p_bc(lat_w<float>(0)), K)), both);
  pair(1, 3, ux, dux, sx, lat_w<float>(1));
  pair(2, 4, uy, duy, sy, lat_w<float>(2));
  pair(5, 7, p_add(ux, uy), p_add(dux, duy), p_add(sx, sy), lat_w<float>(5));
  pair(6, 8, p_sub(uy, ux), p_sub(duy, dux), p_sub(sy, sx), lat_w<float>(6));
}

// Eq. 16 with g^eq of Eq. 18 and the source phi (second Eq. 19) for two nodes.
__device__ __forceinline__ void pair_collide_g(const float2 (&gs)[9], float* __restrict__ go, int plane, bool both,
                                               float2 T, float2 dT, float2 uax, float2 uay, float2 phi,
                                               float omega) {
  const float2 om = p_bc(omega);
  const float2 usq = p_fma(uax, uax, p_mul(uay, uay));
  const float2 Kg = p_fma(om, p_fma(p_mul(p_bc(-1.5f), T), usq, dT), phi);
  const float2 t45 = p_mul(p_bc(4.5f * omega), T), t3 = p_mul(p_bc(3.0f * omega), T), keep = p_bc(1.0f - omega);
  auto pair = [&](int i, int j, float2 cu, float w) {
    const float2 wv = p_bc(w);
    const float2 sym = p_mul(wv, p_fma(p_mul(t45, cu), cu, Kg));
    const float2 anti = p_mul(p_mul(wv, t3), cu);
    pair_store(go + i * plane, p_add(p_fma(keep, gs[i], sym), anti), both);
    pair_store(go + j * plane, p_sub(p_fma(keep, gs[j], sym), anti), both);
  };
  pair_store(go, p_fma(keep, gs[0], p_mul(p_bc(lat_w<float>(0)), Kg)), both);
  pair(1, 3, uax, lat_w<float>(1));
  pair(2, 4, uay, lat_w<float>(2));
  pair(5, 7, p_add(uax, uay), lat_w<float>(5));
  pair(6, 8, p_sub(uay, uax), lat_w<float>(6));
}

// Asynchronous copy of 8 bytes (two adjacent FP32 populations).
__device__ __forceinline__ void cp_async_pair(float2* smem, const float* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}

// Pull of the populations of the nodes (x, x + 1) of row rn into this thread's ring
// slot (9 float2 at stride `stride`): element copies per lane, 8-byte copies where the
// two sources are adjacent and aligned.  Wall links take the node's own opposite
// population (halfway bounce-back); links from outside an open end are left for the
// boundary fill; lanes outside the domain get nothing.
template <bool THERMAL>
__device__ __forceinline__ void pair_pull(float2* f_dst, float2* g_dst, int stride, const float* __restrict__ Fin,
                                          const float* __restrict__ Gin, int plane, int pitch, int x, int rn, int nx,
                                          int ny, bool perx, bool pery, bool local, bool wlo, bool whi, bool top,
                                          InstState* bst) {
  const long long nbuf = 9LL * plane;  // elements of one population buffer (bounds checks)
  const bool interior = !local && x >= 1 && x + 2 <= nx - 1 && rn >= 1 && rn <= ny - 2;
  if (interior) {
    const int node = rn * pitch + x;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int off = node + i * plane - lat_cy(i) * pitch - lat_cx(i);
      if (!idx_ok(bst, off, nbuf) || !idx_ok(bst, off + 1, nbuf)) continue;
      if (lat_cx(i) == 0) {
        cp_async_pair(f_dst + i * stride, Fin + off);
        if (THERMAL) cp_async_pair(g_dst + i * stride, Gin + off);
      } else {
        float* fd = reinterpret_cast<float*>(f_dst + i * stride);
        cp_async_elem(fd, Fin + off);
        cp_async_elem(fd + 1, Fin + off + 1);
        if (THERMAL) {
          float* gd = reinterpret_cast<float*>(g_dst + i * stride);
          cp_async_elem(gd, Gin + off);
          cp_async_elem(gd + 1, Gin + off + 1);
        }
      }
    }
    return;
  }
#pragma unroll
  for (int lane = 0; lane < 2; ++lane) {
    int xl = x + lane;
    if (perx) xl = wrap_index(xl, nx);
    if (xl < 0 || xl >= nx) continue;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int cxi = local ? 0 : lat_cx(i), cyi = local ? 0 : lat_cy(i);
      int src, pl = i;
      const bool wall = !local && ((cyi == 1 && wlo) || (cyi == -1 && whi));
      if (wall) {
        src = rn * pitch + xl;
        pl = lat_opp(i);
      } else {
        int sx = xl - cxi, sy = rn - cyi;
        if (perx) sx = wrap_index(sx, nx);
        if (pery) sy = wrap_index(sy, ny);
        if (sx < 0 || sx >= nx || (top && cyi == -1)) continue;  // unknown link at an open end
        src = sy * pitch + sx;
      }
      if (!idx_ok(bst, pl * plane + src, nbuf)) continue;
      cp_async_elem(reinterpret_cast<float*>(f_dst + i * stride) + lane, Fin + pl * plane + src);
      if (THERMAL) cp_async_elem(reinterpret_cast<float*>(g_dst + i * stride) + lane, Gin + pl * plane + src);
    }
  }
}

template <bool THERMAL, int B>
constexpr size_t pair_smem_bytes() {
  return sizeof(float2) * (size_t)B * (9 * F_SLOTS + (THERMAL ? 9 * G_SLOTS : 0)) +
         sizeof(float) * (size_t)(2 * B) * 9;
}

template <bool THERMAL, int B>
__global__ void __launch_bounds__(B, (B <= 32 ? 12 : (B <= 64 ? 6 : 3)))
lbm_pair_kernel(const Inst* __restrict__ insts, const Tile* __restrict__ tiles) {
  constexpr int NC = 2 * B;     // columns of the psi / u_act rings
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  float2* const sF = reinterpret_cast<float2*>(dyn_smem);         // [F_SLOTS][9][B]
  float2* const sG = sF + F_SLOTS * 9 * B;                        // [G_SLOTS][9][B]
  float* const sPsi = reinterpret_cast<float*>(sG + (THERMAL ? G_SLOTS * 9 * B : 0));  // [3][NC]
  float* const sUx = sPsi + 3 * NC;                               // [3][NC]
  float* const sUy = sUx + 3 * NC;                                // [3][NC]
  __shared__ Inst sI;
  __shared__ KConst<float> sC;
  __shared__ double sRed[B / 32 > 0 ? B / 32 : 1][NPART];
  __shared__ int sLast;

  const int tid = threadIdx.x;
  const Tile tile = tiles[blockIdx.x];
  {
    const int* src = reinterpret_cast<const int*>(insts + tile.inst);
    int* dst = reinterpret_cast<int*>(&sI);
    for (int k = tid; k < (int)(sizeof(Inst) / 4); k += B) dst[k] = src[k];
  }
  __syncthreads();
  InstState* st = sI.st;
  const long long step = st->step;
  if (tid == 0) fill_consts<float>(sC, sI, st->rho_avg[(step - 1) & 1]);
  __syncthreads();

  const int nx = sI.nx, ny = sI.ny, pitch = sI.pitch;
  const int plane = (int)sI.plane;
  const bool local = st->local_read != 0;
  const bool perx = sI.geometry != GEOM_CHANNEL;
  const bool pery = sI.geometry == GEOM_PERIODIC;
  const bool channel = sI.geometry == GEOM_CHANNEL;
  const bool pool = sI.geometry == GEOM_POOL;
  const bool multiphase = sI.multiphase != 0;
  const float* __restrict__ Fin = static_cast<const float*>(sI.f[step & 1]);
  const float* __restrict__ Gin = static_cast<const float*>(sI.g[step & 1]);
  float* __restrict__ Fout = static_cast<float*>(sI.f[(step + 1) & 1]);
  float* __restrict__ Gout = static_cast<float*>(sI.g[(step + 1) & 1]);
  const float T0 = sC.T0;

  // this thread's nodes: xa = x0 - 2 + 2 t and xa + 1 (ring columns 2t, 2t + 1)
  const bool active = tid < B - 2;
  const int t = active ? tid : 0;
  const int xa = tile.x0 - 2 + 2 * t;
  const int xn0 = perx ? wrap_index(xa, nx) : xa;
  const int xn1 = perx ? wrap_index(xa + 1, nx) : xa + 1;
  const bool in0 = active && (perx || (xa >= 0 && xa < nx));
  const bool in1 = active && (perx || (xa + 1 >= 0 && xa + 1 < nx));
  const bool out_thread = tid >= 1 && tid <= B - 4 && xa < nx;  // outputs [x0, x0 + W)
  const bool out1 = out_thread && xa + 1 < nx;                    // second lane inside too
  const bool f_thread = active;  // u_act needed on columns x0 - 1 .. x0 + W (lane 1 of thread 0 on)
  // ring columns of the W / E neighbours of each lane; at an open end the ghost
  // column repeats the end column
  const int c0 = 2 * t, c1 = 2 * t + 1;
  const int iW0 = (!perx && xa == 0) ? c0 : c0 - 1;
  const int iE0 = (!perx && xa == nx - 1) ? c0 : c1;
  const int iW1 = c0;
  const int iE1 = (!perx && xa + 1 == nx - 1) ? c1 : c1 + 1;
  const bool edge = channel && (xa <= 0 || xa + 1 >= nx - 1);  // a lane at the inlet or outlet
  const float2 lane_mask = make_float2(1.0f, out1 ? 1.0f : 0.0f);

  const int nrow = tile.y1 - tile.y0;
  const int kend = nrow + 4;

  auto issue_row = [&](int k, int fslot, int gslot) {
    if (active && k < kend) {
      const int r = tile.y0 - 2 + k;
      if (pery || (r >= 0 && r < ny)) {
        const int rn = pery ? wrap_index(r, ny) : r;
        pair_pull<THERMAL>(sF + fslot * 9 * B + t, sG + gslot * 9 * B + t, B, Fin, Gin, plane, pitch, xa, rn, nx, ny,
                           perx, pery, local, !pery && rn == 0, !pery && !pool && rn == ny - 1,
                           pool && rn == ny - 1, st);
      }
    }
    cp_async_commit();
  };

  float2 acc_m = p_bc(0.0f), acc_e = p_bc(0.0f);
  float acc_h = 0.0f, acc_fi = 0.0f, acc_fo = 0.0f, acc_va = 0.0f, acc_wv = 0.0f, acc_hv = 0.0f, acc_zv = 0.0f;
  const int zlo = sI.heater_x0 - sI.heater_len, zhi = sI.heater_x0 + 2 * sI.heater_len;
  float2 rho_p = p_bc(1.0f), drho_p = p_bc(0.0f), ux_p = p_bc(0.0f), uy_p = p_bc(0.0f), T_p = p_bc(T0),
         dT_p = p_bc(0.0f), coef_p = p_bc(0.0f);
  float2 T_p2 = p_bc(T0), dT_p2 = p_bc(0.0f), coef_p2 = p_bc(0.0f);

  int f_cur = 0, g_cur = 0;
  issue_row(0, f_cur, g_cur);
  for (int k = 0; k < kend; ++k) {
    const int r = tile.y0 - 2 + k;
    const int f_next = (f_cur == F_SLOTS - 1) ? 0 : f_cur + 1;
    const int f_prev = (f_cur == 0) ? F_SLOTS - 1 : f_cur - 1;
    const int f_prev2 = (f_prev == 0) ? F_SLOTS - 1 : f_prev - 1;
    const int g_next = (g_cur + 1) & (G_SLOTS - 1);
    const int g_prev2 = (g_cur + 2) & (G_SLOTS - 1);
    issue_row(k + 1, f_next, g_next);
    cp_async_wait_1();

    // ===================== phase A: row r =====================
    const bool row_ok = pery || (r >= 0 && r < ny);
    const int rn = pery ? wrap_index(r, ny) : r;
    PairState ns;
    ns.rho = p_bc(1.0f); ns.drho = p_bc(0.0f); ns.ux = p_bc(0.0f); ns.uy = p_bc(0.0f);
    ns.T = p_bc(T0); ns.dT = p_bc(0.0f); ns.coef = p_bc(0.0f); ns.dpsi = p_bc(0.0f);
    if (active && row_ok) {
      float2* fs = sF + f_cur * 9 * B + t;
      float2* gs = sG + g_cur * 9 * B + t;
      float2 fc[9], gc[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        fc[i] = fs[i * B];
        gc[i] = THERMAL ? gs[i * B] : p_bc(0.0f);
      }
      const bool wlo = !pery && rn == 0, whi = !pery && !pool && rn == ny - 1, top = pool && rn == ny - 1;
      if (!local && (wlo || whi || edge || top)) {
        // boundary nodes: the scalar boundary fill, lane by lane, written back to the ring
#pragma unroll
        for (int lane = 0; lane < 2; ++lane) {
          const int xl = lane ? xn1 : xn0;
          if (!(lane ? in1 : in0)) continue;
          const NodeBC nb{wlo, whi, channel && xl == 0, channel && xl == nx - 1, top};
          if (!(nb.wlo || nb.whi || nb.inl || nb.outl || nb.top)) continue;
          float f1[9], g1[9];
#pragma unroll
          for (int i = 0; i < 9; ++i) {
            f1[i] = lane ? fc[i].y : fc[i].x;
            g1[i] = lane ? gc[i].y : gc[i].x;
          }
          boundary_fill<float, THERMAL>(f1, g1, nb, sI, sC, Gin, plane, pitch, rn * pitch + xl, xl, perx, step);
#pragma unroll
          for (int i = 0; i < 9; ++i) {
            if (lane) {
              fc[i].y = f1[i];
              gc[i].y = g1[i];
            } else {
              fc[i].x = f1[i];
              gc[i].x = g1[i];
            }
            fs[i * B] = fc[i];
            if (THERMAL) gs[i * B] = gc[i];
          }
        }
      }
      ns = pair_state<THERMAL>(fc, gc, sC, multiphase);
      if ((in0 && ns.bad0) || (in1 && ns.bad1)) atomicOr(&st->status, STATUS_UNSTABLE);
      *reinterpret_cast<float2*>(sPsi + f_cur * NC + c0) = ns.dpsi;
      const bool out_row = r >= tile.y0 && r < tile.y1;
      if (out_thread && out_row) {
        acc_m = p_fma(ns.drho, lane_mask, acc_m);
        if (THERMAL) {
          acc_e = p_fma(ns.dT, lane_mask, acc_e);
          if (wlo) {
            if (xn0 >= sI.heater_x0 && xn0 < sI.heater_x0 + sI.heater_len) acc_h += ns.dT.x;
            if (out1 && xn1 >= sI.heater_x0 && xn1 < sI.heater_x0 + sI.heater_len) acc_h += ns.dT.y;
          }
        }
        if (sI.bubble_stats) {
          const float v0 = ns.drho.x < sC.drho_vapor ? 1.0f : 0.0f;
          const float v1 = (out1 && ns.drho.y < sC.drho_vapor) ? 1.0f : 0.0f;
          acc_va += v0 + v1;
          if (xn0 >= zlo && xn0 < zhi) acc_zv += v0;
          if (xn1 >= zlo && xn1 < zhi) acc_zv += v1;
          if (wlo) {
            acc_wv += v0 + v1;
            if (xn0 >= sI.heater_x0 && xn0 < sI.heater_x0 + sI.heater_len) acc_hv += v0;
            if (xn1 >= sI.heater_x0 && xn1 < sI.heater_x0 + sI.heater_len) acc_hv += v1;
          }
        }
        if (channel && rn == ny / 2) {
          if (xn0 == 1) st->p_probe[2 * (step & 1)] = (double)ns.p.x;
          if (out1 && xn1 == 1) st->p_probe[2 * (step & 1)] = (double)ns.p.y;
          if (xn0 == nx - 2) st->p_probe[2 * (step & 1) + 1] = (double)ns.p.x;
          if (out1 && xn1 == nx - 2) st->p_probe[2 * (step & 1) + 1] = (double)ns.p.y;
          __threadfence();
        }
      }
    }
    __syncthreads();

    // ===================== phase B: row q = r - 1 =====================
    const int q = r - 1;
    if (q >= tile.y0 - 1 && f_thread && (pery || (q >= 0 && q < ny))) {
      const bool sol_m = !pery && q == 0;
      const bool sol_p = !pery && !pool && q == ny - 1;
      float2 Fx = p_bc(0.0f), Fy = p_bc(0.0f);
      if (multiphase) {
        const float* P0 = sPsi + f_prev * NC;
        const float* Pp = (pool && q == ny - 1) ? P0 : sPsi + f_cur * NC;  // pool top: ghost row
        const float* Pm = sPsi + f_prev2 * NC;
        const float2 zc = p_bc(0.0f);
        const float2 dc = *reinterpret_cast<const float2*>(P0 + c0);
        const float2 dE = make_float2(P0[iE0], P0[iE1]), dW = make_float2(P0[iW0], P0[iW1]);
        float2 dN = zc, dNE = zc, dNW = zc, dS = zc, dSE = zc, dSW = zc;
        if (!sol_p) {
          dN = *reinterpret_cast<const float2*>(Pp + c0);
          dNE = make_float2(Pp[iE0], Pp[iE1]);
          dNW = make_float2(Pp[iW0], Pp[iW1]);
        }
        if (!sol_m) {
          dS = *reinterpret_cast<const float2*>(Pm + c0);
          dSE = make_float2(Pm[iE0], Pm[iE1]);
          dSW = make_float2(Pm[iW0], Pm[iW1]);
        }
        pair_force(dc, dE, dW, dN, dNE, dNW, dS, dSE, dSW, sol_m, sol_p, sC, Fx, Fy);
      }
      Fy = p_sub(Fy, p_mul(p_add(drho_p, p_bc(sC.rho_ref_minus_avg)), p_bc(sC.g_a)));  // Eq. 14
      const float2 inv_rho = p_rcp(rho_p);
      const float2 dux = p_mul(Fx, inv_rho), duy = p_mul(Fy, inv_rho);
      const float2 uax = p_fma(p_bc(0.5f), dux, ux_p), uay = p_fma(p_bc(0.5f), duy, uy_p);  // Eq. 7
      *reinterpret_cast<float2*>(sUx + f_prev * NC + c0) = uax;
      *reinterpret_cast<float2*>(sUy + f_prev * NC + c0) = uay;
      if (out_thread && q >= tile.y0 && q < tile.y1) {
        const float2* fsp = sF + f_prev * 9 * B + t;
        float2 fsv[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) fsv[i] = fsp[i * B];
        // the nine stores go to q * pitch + xa + i * plane (+ 1 for the second node): checking the
        // first and the last covers them all in a bounds-checked build
        if (idx_ok(st, q * pitch + xa, 9LL * plane) && idx_ok(st, q * pitch + xa + 8LL * plane + out1, 9LL * plane))
          pair_collide_f(fsv, Fout + (q * pitch + xa), plane, out1, rho_p, drho_p, ux_p, uy_p, dux, duy, sC.omega_f);
        if (edge) {
          if (xn0 == 0) acc_fi += rho_p.x * uax.x;
          if (xn0 == nx - 1) acc_fo += rho_p.x * uax.x;
          if (out1 && xn1 == nx - 1) acc_fo += rho_p.y * uax.y;
        }
      }
    }
    __syncthreads();

    // ===================== phase C: row q2 = r - 2 =====================
    if (THERMAL) {
      const int q2 = r - 2;
      if (out_thread && q2 >= tile.y0 && q2 < tile.y1) {
        const float* Ux = sUx + f_prev2 * NC;
        const float2 uxE = make_float2(Ux[iE0], Ux[iE1]), uxW = make_float2(Ux[iW0], Ux[iW1]);
        const float2 uyC = *reinterpret_cast<const float2*>(sUy + f_prev2 * NC + c0);
        const float2 uyN = (pool && q2 == ny - 1) ? uyC : *reinterpret_cast<const float2*>(sUy + f_prev * NC + c0);
        const float2 uyS = *reinterpret_cast<const float2*>(sUy + f_cur * NC + c0);  // slot of row r-3
        const bool wall_lo = !pery && q2 == 0, wall_hi = !pery && !pool && q2 == ny - 1;
        float2 dyu = p_mul(p_bc(0.5f), p_sub(uyN, uyS));
        if (wall_lo || wall_hi) dyu = (wall_lo && wall_hi) ? p_bc(0.0f) : (wall_lo ? p_sub(uyN, uyC) : p_sub(uyC, uyS));
        const float2 divu = p_fma(p_bc(0.5f), p_sub(uxE, uxW), dyu);
        const float2* gsp = sG + g_prev2 * 9 * B + t;
        float2 gsv[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) gsv[i] = gsp[i * B];
        const float2 uax = *reinterpret_cast<const float2*>(Ux + c0);
        if (idx_ok(st, q2 * pitch + xa, 9LL * plane) && idx_ok(st, q2 * pitch + xa + 8LL * plane + out1, 9LL * plane))
          pair_collide_g(gsv, Gout + (q2 * pitch + xa), plane, out1, T_p2, dT_p2, uax, uyC, p_mul(coef_p2, divu),
                         sC.omega_g);
      }
    }

    T_p2 = T_p;
    dT_p2 = dT_p;
    coef_p2 = coef_p;
    rho_p = ns.rho;
    drho_p = ns.drho;
    ux_p = ns.ux;
    uy_p = ns.uy;
    T_p = ns.T;
    dT_p = ns.dT;
    coef_p = ns.coef;
    f_cur = f_next;
    g_cur = g_next;
  }

  // ---------------- per-tile partials into the launch's totals ----------------
  double acc[NPART] = {(double)acc_m.x + (double)acc_m.y, (double)acc_e.x + (double)acc_e.y, (double)acc_h,
                       (double)acc_fi, (double)acc_fo, (double)acc_va, (double)acc_wv, (double)acc_hv,
                       (double)acc_zv};
  post_partials<B, THERMAL, MODE_STEP>(sI, st, tile, acc, sRed, &sLast, step);
}

template <bool THERMAL, int B>
cudaError_t launch_pair_one(const Inst* d_inst, const Tile* d_tiles, int ntiles, cudaStream_t s) {
  constexpr size_t smem = pair_smem_bytes<THERMAL, B>();
  static unsigned long long configured = 0ull;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(configured & bit)) {
    e = cudaFuncSetAttribute(lbm_pair_kernel<THERMAL, B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured |= bit;
  }
  lbm_pair_kernel<THERMAL, B><<<ntiles, B, smem, s>>>(d_inst, d_tiles);
  return cudaGetLastError();
}

template <bool THERMAL, int B>
int resident_pair_one() {
  constexpr size_t smem = pair_smem_bytes<THERMAL, B>();
  auto fn = lbm_pair_kernel<THERMAL, B>;
  int n = 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, B, smem) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

inline int resident_pair(int thermal, int cols) {
  if (thermal) {
    switch (cols) {
      case 64: return resident_pair_one<true, 32>();
      case 128: return resident_pair_one<true, 64>();
      case 256: return resident_pair_one<true, 128>();
    }
  } else {
    switch (cols) {
      case 64: return resident_pair_one<false, 32>();
      case 128: return resident_pair_one<false, 64>();
      case 256: return resident_pair_one<false, 128>();
    }
  }
  return 1;
}

// The packed step for a tile table built for `cols` columns (cols / 2 threads).
inline cudaError_t launch_pair(int thermal, int cols, const Inst* d_inst, const Tile* d_tiles, int ntiles,
                               cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  if (thermal) {
    switch (cols) {
      case 64: return launch_pair_one<true, 32>(d_inst, d_tiles, ntiles, s);
      case 128: return launch_pair_one<true, 64>(d_inst, d_tiles, ntiles, s);
      case 256: return launch_pair_one<true, 128>(d_inst, d_tiles, ntiles, s);
    }
  } else {
    switch (cols) {
      case 64: return launch_pair_one<false, 32>(d_inst, d_tiles, ntiles, s);
      case 128: return launch_pair_one<false, 64>(d_inst, d_tiles, ntiles, s);
      case 256: return launch_pair_one<false, 128>(d_inst, d_tiles, ntiles, s);
    }
  }
  return cudaErrorInvalidValue;
}

}  // namespace pplbm
