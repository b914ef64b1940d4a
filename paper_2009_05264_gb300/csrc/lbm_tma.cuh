// FP32 fused step with its populations staged by the Tensor Memory Accelerator.
//
// Same time step as lbm_fused_kernel (Sec. 2 of Mukherjee, Basu & Mondal, arXiv
// 2009.05264, boundary conditions of Sec. 2.C), lean form, 128 threads per CTA.  The
// scalar kernel stages, per thread, the 18 populations its node pulls, with one
// 4-byte cp.async each (18 copies and their address arithmetic per node).  Here the CTA
// stages, per row, the 128 columns [x0 - 4, x0 + 124) of each population plane i taken
// from row r - c_iy into a shared-memory row of a ring; the pull's shift along x is then
// a constant offset of the shared-memory read (node x of plane i sits at position
// x - x0 + 4 - c_ix).  One thread issues one bulk tensor copy (cp.async.bulk.tensor.3d)
// per plane-row; completion is one mbarrier per ring slot (expect-tx of the 9 boxes'
// bytes), and every thread waits on the slot's barrier (bounded).
//
// Nodes whose pull leaves the staged box or needs a boundary condition (the two
// outermost rows and columns of the lattice, periodic wrap-around, and the first step
// after an initialisation, whose buffer holds post-stream populations) are "special":
// their thread pulls them with plain loads as the scalar kernel does, completes them
// with boundary_fill, and writes the result back into its own positions of the staged
// rows (one position per plane per node, so no two threads write the same element),
// then fences its generic-proxy writes before the slot is refilled by the async proxy.
//
// Ring slots: f of rows r + 1 (in flight), r and r - 1 (3 slots); g of rows r + 1 down
// to r - 3 (5 slots).  Row r + 1 is issued at the top of iteration r with no barrier
// since the previous iteration's phase C, which still reads g of row r - 3, so that slot
// must not be the one refilled.  Every mbarrier wait is bounded; a wait that gives up sets STATUS_TIMEOUT, the CTA leaves the row loop, drains its copies in
// flight (again bounded) and still posts its partials, so the launch ends and the host
// reports LBM_ETIMEOUT.
#pragma once

#include "lbm_kernels.cuh"

namespace pplbm {

constexpr int ST_COLS = 128;                             // threads per CTA and columns per staged row
constexpr int ST_FS = 3;                                 // f ring slots
constexpr int ST_GS = 5;                                 // g ring slots
constexpr int ST_RW = 9 * ST_COLS;                       // floats per staged row of one population set
constexpr unsigned ST_ROW_BYTES = ST_RW * sizeof(float); // bytes of one row of one population set
constexpr long long TMA_WAIT_LIMIT = 1ll << 22;          // polls of a bounded mbarrier wait

template <bool THERMAL>
constexpr size_t tma_smem_bytes() {
  // 128 bytes of slack to align the rings to 128 bytes
  return 128 + sizeof(float) * ((size_t)ST_RW * (ST_FS + (THERMAL ? ST_GS : 0)) + 9 * (ST_COLS - 4));
}

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// Make the initialised barriers visible to the async proxy (the tensor copies).
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Test, without waiting, whether the phase of the given parity has completed.
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// The row waits under a test's poll cap: at most `polls` non-blocking tests (a blocking try_wait
// may suspend the thread until the copies land, so one poll of it rarely gives up).
__device__ __forceinline__ bool mbar_poll(unsigned long long* bar, unsigned parity, unsigned polls) {
  for (unsigned it = 0; it < polls; ++it)
    if (mbar_test(bar, parity)) return true;
  return false;
}
// Wait for the phase of the given parity to complete; false if it has not after `limit`
// polls of the (potentially blocking) try_wait.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, long long limit = TMA_WAIT_LIMIT) {
  const unsigned a = smem_u32(bar);
  for (long long it = 0; it < limit; ++it) {
    unsigned done;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// One 3-D tensor box (x, y, z) -> shared memory, completing on `bar`.  x must be a
// multiple of 4 (16 bytes of FP32); y and z may lie outside the tensor (zero fill).
__device__ __forceinline__ void tma_load_3d(float* dst, const void* tmap, int x, int y, int z,
                                            unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(tmap)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
// Order this thread's generic-proxy shared-memory writes before later async-proxy
// (tensor copy) writes to the same addresses.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// The pulled populations of one node in a staged row: plane i at the node's column
// shifted by -c_ix (row points at the node's unshifted position in plane 0).
struct ShiftedPops {
  const float* row;
  __device__ __forceinline__ float operator()(int i) const { return row[i * ST_COLS - lat_cx(i)]; }
};

// Plain-load pull of one node (the scalar kernel's pull, synchronous): interior and
// periodic links from the neighbour, wall links from the node's own opposite
// population (also at the corners where a wall meets an open end), the other links
// from outside an open end left at zero for boundary_fill.
template <bool THERMAL>
__device__ __forceinline__ void pull_direct(float (&fc)[9], float (&gc)[9], const float* __restrict__ Fin,
                                            const float* __restrict__ Gin, int plane, int pitch, int xn, int rn,
                                            int nx, int ny, bool perx, bool pery, bool local, const NodeBC& nb,
                                            InstState* bst) {
  const int node = rn * pitch + xn;
  const long long nbuf = 9LL * plane;  // elements of one population buffer (bounds checks)
  if (local) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const bool ok = idx_ok(bst, i * plane + node, nbuf);
      fc[i] = ok ? ld_ro(Fin + i * plane + node) : 0.0f;
      gc[i] = THERMAL && ok ? ld_ro(Gin + i * plane + node) : 0.0f;
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
    // at a corner of a wall and an open end the wall's bounce-back takes the link
    const bool unknown = !wall && ((cxi == 1 && nb.inl) || (cxi == -1 && nb.outl));
    fc[i] = 0.0f;
    gc[i] = 0.0f;
    if (unknown) continue;
    int src = node, pl = lat_opp(i);
    if (!wall) {
      src = (cyi == 1 ? rm : (cyi == -1 ? rp : rn)) * pitch + (cxi == 1 ? xm : (cxi == -1 ? xp : xn));
      pl = i;
    }
    if (!idx_ok(bst, pl * plane + src, nbuf)) continue;
    fc[i] = ld_ro(Fin + pl * plane + src);
    if (THERMAL) gc[i] = ld_ro(Gin + pl * plane + src);
  }
}

// Lean FP32 step (no pool geometry, Hazi-Markus source or bubble counters), one step of
// every tile of the launch.  Tiles must be 120 columns wide (x0 a multiple of 120) and each
// instance must carry its four tensor maps (f and g, both buffers).  PCONST: the launch
// covers one instance whose descriptor and converted constants arrive as the kernel
// parameter kp (as in lbm_fused_kernel).
template <bool THERMAL, bool PCONST>
__global__ void __launch_bounds__(ST_COLS, 5)
lbm_tma_kernel(const Inst* __restrict__ insts, const Tile* __restrict__ tiles, unsigned max_polls,
               const __grid_constant__ KParams<float> kp) {
  constexpr int B = ST_COLS;
  constexpr int W = out_cols<B>();
  constexpr int NS = B - 4;
  extern __shared__ unsigned char tma_dyn_smem[];
  float* const sF =
      reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(tma_dyn_smem) + 127) & ~uintptr_t(127));  // [FS][9][B]
  float* const sG = sF + ST_FS * ST_RW;                    // [GS][9][B]
  float* const sPsi = sG + (THERMAL ? ST_GS * ST_RW : 0);  // [3][NS]
  float* const sUx = sPsi + 3 * NS;
  float* const sUy = sUx + 3 * NS;
  __shared__ __align__(8) unsigned long long fbar[ST_FS];
  __shared__ __align__(8) unsigned long long gbar[ST_GS];
  __shared__ Inst sI;
  __shared__ KConst<float> sCv;
  __shared__ float sRra;  // rho_ref - rho_avg of the previous step (buoyancy, Eq. 14)
  __shared__ double sRed[B / 32][NPART];
  __shared__ int sLast;
  __shared__ int sAbort;

  const int tid = threadIdx.x;
  const Tile tile = tiles[blockIdx.x];
  if (!PCONST) {
    const int* src = reinterpret_cast<const int*>(insts + tile.inst);
    int* dst = reinterpret_cast<int*>(&sI);
    for (int k = tid; k < (int)(sizeof(Inst) / 4); k += B) dst[k] = src[k];
    __syncthreads();
  }
  const Inst& I = PCONST ? kp.I : sI;
  InstState* st = I.st;
  const long long step = st->step;
  const bool local = st->local_read != 0;
  if (tid == 0) {
    const double rho_avg_prev = st->rho_avg[(step - 1) & 1];
    if (!PCONST) fill_consts<float>(sCv, I, rho_avg_prev);
    sRra = float(I.rho_ref - rho_avg_prev);
    sAbort = 0;
    for (int j = 0; j < ST_FS; ++j) mbar_init(&fbar[j], 1);
    for (int j = 0; j < ST_GS; ++j) mbar_init(&gbar[j], 1);
    mbar_init_fence();
  }
  __syncthreads();
  const KConst<float>& C = PCONST ? kp.C : sCv;

  const int nx = I.nx, ny = I.ny, pitch = I.pitch;
  const int plane = (int)I.plane;
  const bool perx = I.geometry != GEOM_CHANNEL;
  const bool pery = I.geometry == GEOM_PERIODIC;
  const bool channel = I.geometry == GEOM_CHANNEL;
  const bool multiphase = I.multiphase != 0;
  const float* __restrict__ Fin = static_cast<const float*>(I.f[step & 1]);
  const float* __restrict__ Gin = static_cast<const float*>(I.g[step & 1]);
  float* __restrict__ Fout = static_cast<float*>(I.f[(step + 1) & 1]);
  float* __restrict__ Gout = static_cast<float*>(I.g[(step + 1) & 1]);
  const float T0 = C.T0;

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
  const int sm = (!perx && xc == 0) ? s : s - 1;
  const int sp = (!perx && xc == nx - 1) ? s : s + 1;
  const bool inl = channel && xn == 0;
  const bool outl = channel && xn == nx - 1;
  // columns whose pull stays inside the staged row and needs no boundary condition
  const bool col_plain = !local && xc >= 1 && xc <= nx - 2;

  const int nrow = tile.y1 - tile.y0;
  const int kend = nrow + 4;
  const int xbox = tile.x0 - 4;  // first column of every staged row (16-byte aligned)

  // Row k (f, and g when thermal) into ring slots fsl / gsl (thread 0): nine boxes per
  // population set, one barrier per set.
  auto issue_row = [&](int k, int fsl, int gsl) {
    const int r = tile.y0 - 2 + k;
    const unsigned char* tm = static_cast<const unsigned char*>(I.tmaps);
    const void* fmap = tm + 128 * (step & 1);  // f of buffers 0 and 1, then g (128 bytes each)
    const void* gmap = tm + 128 * (2 + (step & 1));
    mbar_arrive_expect_tx(&fbar[fsl], ST_ROW_BYTES);
#pragma unroll
    for (int i = 0; i < 9; ++i) tma_load_3d(sF + fsl * ST_RW + i * B, fmap, xbox, r - lat_cy(i), i, &fbar[fsl]);
    if (THERMAL) {
      mbar_arrive_expect_tx(&gbar[gsl], ST_ROW_BYTES);
#pragma unroll
      for (int i = 0; i < 9; ++i) tma_load_3d(sG + gsl * ST_RW + i * B, gmap, xbox, r - lat_cy(i), i, &gbar[gsl]);
    }
  };

  float acc_m = 0.0f, acc_e = 0.0f, acc_h = 0.0f, acc_fi = 0.0f, acc_fo = 0.0f;
  float rho_p = 1.0f, drho_p = 0.0f, ux_p = 0.0f, uy_p = 0.0f, T_p = T0, dT_p = 0.0f, coef_p = 0.0f;
  float T_p2 = T0, dT_p2 = 0.0f, coef_p2 = 0.0f;

  // ring slots of row k: psi / u (mod 3), staged f (mod ST_FS) and g (mod ST_GS), with the
  // parities of the f and g barrier phases (row k's phase of slot k mod n is (k / n) & 1)
  int p_cur = 0, f_cur = 0, g_cur = 0;
  unsigned f_par = 0u, g_par = 0u;
  if (!local && tid == 0) issue_row(0, 0, 0);
  int k = 0;
  for (; k < kend; ++k) {
    const int r = tile.y0 - 2 + k;
    const int p_prev = (p_cur == 0) ? 2 : p_cur - 1;     // row r - 1
    const int p_prev2 = (p_prev == 0) ? 2 : p_prev - 1;  // row r - 2 (and r + 1)
    const int f_prev = (f_cur == 0) ? ST_FS - 1 : f_cur - 1;
    const int g_prev2 = (g_cur >= 2) ? g_cur - 2 : g_cur + ST_GS - 2;
    if (!local && tid == 0 && k + 1 < kend)
      issue_row(k + 1, f_cur == ST_FS - 1 ? 0 : f_cur + 1, g_cur == ST_GS - 1 ? 0 : g_cur + 1);
    if (!local) {
      bool ok = max_polls ? mbar_poll(&fbar[f_cur], f_par, max_polls) : mbar_wait(&fbar[f_cur], f_par);
      if (THERMAL) ok = (max_polls ? mbar_poll(&gbar[g_cur], g_par, max_polls) : mbar_wait(&gbar[g_cur], g_par)) && ok;
      if (!ok) {
        atomicOr(&st->status, STATUS_TIMEOUT);
        sAbort = 1;
      }
    }

    // ===================== phase A: row r =====================
    const bool row_ok = pery || (r >= 0 && r < ny);
    const int rn = pery ? wrap_index(r, ny) : r;
    NodeState<float> ns;
    ns.rho = 1.0f; ns.drho = 0.0f; ns.ux = 0.0f; ns.uy = 0.0f;
    ns.T = T0; ns.dT = 0.0f; ns.coef = 0.0f; ns.dpsi = 0.0f;
    if (col_ok && row_ok) {
      float* const fs = sF + f_cur * ST_RW + (s + 2);
      float* const gs = sG + g_cur * ST_RW + (s + 2);
      float fc[9], gc[9];
      const bool plain = col_plain && r >= 1 && r <= ny - 2;
      if (plain) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          fc[i] = fs[i * B - lat_cx(i)];
          gc[i] = THERMAL ? gs[i * B - lat_cx(i)] : 0.0f;
        }
      } else {
        const NodeBC nb{!pery && rn == 0, !pery && rn == ny - 1, inl, outl, false};
        pull_direct<THERMAL>(fc, gc, Fin, Gin, plane, pitch, xn, rn, nx, ny, perx, pery, local, nb, I.st);
        if (!local && (nb.wlo || nb.whi || inl || outl))
          boundary_fill<float, THERMAL>(fc, gc, nb, I, C, Gin, plane, pitch, rn * pitch + xn, xn, perx, step);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          fs[i * B - lat_cx(i)] = fc[i];
          if (THERMAL) gs[i * B - lat_cx(i)] = gc[i];
        }
        fence_proxy_async_smem();
      }
      ns = node_state<float, THERMAL>(fc, gc, C, multiphase, false);
      if (ns.bad) atomicOr(&st->status, STATUS_UNSTABLE);
      sPsi[p_cur * NS + s] = ns.dpsi;
      const bool out_row = r >= tile.y0 && r < tile.y1;
      if (out_col && out_row) {
        acc_m += ns.drho;
        if (THERMAL) {
          acc_e += ns.dT;
          if (!pery && rn == 0 && xn >= I.heater_x0 && xn < I.heater_x0 + I.heater_len) acc_h += ns.dT;
        }
        if (channel && rn == ny / 2 && (xn == 1 || xn == nx - 2)) {
          if (xn == 1) st->p_probe[2 * (step & 1)] = (double)ns.p;
          if (xn == nx - 2) st->p_probe[2 * (step & 1) + 1] = (double)ns.p;
          __threadfence();
        }
      }
    }
    __syncthreads();
    if (sAbort) break;

    // ===================== phase B: row q = r - 1 =====================
    const int q = r - 1;
    if (q >= tile.y0 - 1 && f_col && (pery || (q >= 0 && q < ny))) {
      const bool sol_m = !pery && q == 0;
      const bool sol_p = !pery && q == ny - 1;
      float Fx = 0.0f, Fy = 0.0f;
      if (multiphase) {
        const float* P0 = sPsi + p_prev * NS;
        const float* Pp = sPsi + p_cur * NS;
        const float* Pm = sPsi + p_prev2 * NS;
        sc_force<float>(P0[s], P0[sp], P0[sm], sol_p ? 0.0f : Pp[s], sol_p ? 0.0f : Pp[sp], sol_p ? 0.0f : Pp[sm],
                        sol_m ? 0.0f : Pm[s], sol_m ? 0.0f : Pm[sp], sol_m ? 0.0f : Pm[sm], sol_m, sol_p, C, Fx, Fy);
      }
      Fy -= (drho_p + sRra) * C.g_a;  // Eq. 14, gravity along -y
      const float inv_rho = fast_rcp(rho_p);
      const float dux = Fx * inv_rho, duy = Fy * inv_rho;
      const float uax = ux_p + 0.5f * dux, uay = uy_p + 0.5f * duy;  // Eq. 7
      sUx[p_prev * NS + s] = uax;
      sUy[p_prev * NS + s] = uay;
      if (out_col && q >= tile.y0 && q < tile.y1) {
        collide_f<float>(ShiftedPops{sF + f_prev * ST_RW + (s + 2)}, plane_out(Fout, q * pitch + xn, plane, I.st, 9LL * plane),
                         rho_p, drho_p, ux_p, uy_p, dux, duy, C.omega_f);
        if (channel && xn == 0) acc_fi += rho_p * uax;
        if (channel && xn == nx - 1) acc_fo += rho_p * uax;
      }
    }
    __syncthreads();

    // ===================== phase C: row q2 = r - 2 =====================
    if (THERMAL) {
      const int q2 = r - 2;
      if (out_col && q2 >= tile.y0 && q2 < tile.y1) {
        const float uxE = sUx[p_prev2 * NS + sp], uxW = sUx[p_prev2 * NS + sm];
        const float uyN = sUy[p_prev * NS + s];
        const float uyS = sUy[p_cur * NS + s];  // slot of row r - 3
        const bool wall_lo = !pery && q2 == 0, wall_hi = !pery && q2 == ny - 1;
        float dyu = 0.5f * (uyN - uyS);
        if (wall_lo || wall_hi) {
          const float uyC = sUy[p_prev2 * NS + s];
          dyu = (wall_lo && wall_hi) ? 0.0f : (wall_lo ? uyN - uyC : uyC - uyS);
        }
        const float divu = 0.5f * (uxE - uxW) + dyu;
        collide_g<float>(ShiftedPops{sG + g_prev2 * ST_RW + (s + 2)}, plane_out(Gout, q2 * pitch + xn, plane, I.st, 9LL * plane),
                         T_p2, dT_p2, sUx[p_prev2 * NS + s], sUy[p_prev2 * NS + s], coef_p2 * divu, C.omega_g);
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
    p_cur = (p_cur == 2) ? 0 : p_cur + 1;
    if (++f_cur == ST_FS) {
      f_cur = 0;
      f_par ^= 1u;
    }
    if (++g_cur == ST_GS) {
      g_cur = 0;
      g_par ^= 1u;
    }
  }
  if (k < kend && !local && tid == 0) {
    // aborted at row k: let the copies of row k (whose waits gave up, possibly before they
    // landed) and of row k + 1 (issued before them) land before the CTA's shared memory is
    // released (row j: slot j mod depth, parity (j / depth) & 1); each wait has the full limit
    for (int j = k; j <= k + 1 && j < kend; ++j) {
      mbar_wait(&fbar[j % ST_FS], (j / ST_FS) & 1);
      if (THERMAL) mbar_wait(&gbar[j % ST_GS], (j / ST_GS) & 1);
    }
  }

  // ---------------- per-tile partials into the launch's totals ----------------
  double acc[NPART] = {(double)acc_m, (double)acc_e, (double)acc_h, (double)acc_fi, (double)acc_fo, 0.0, 0.0, 0.0, 0.0};
  post_partials<B, THERMAL, MODE_STEP>(I, st, tile, acc, sRed, &sLast, step);
}

template <bool THERMAL, bool PCONST>
cudaError_t launch_tma_t(const Inst* d_inst, const Tile* d_tiles, int ntiles, unsigned max_polls, cudaStream_t s,
                         const KParams<float>& kp) {
  constexpr size_t smem = tma_smem_bytes<THERMAL>();
  auto fn = lbm_tma_kernel<THERMAL, PCONST>;
  static unsigned long long configured = 0ull;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(configured & bit)) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured |= bit;
  }
  fn<<<ntiles, ST_COLS, smem, s>>>(d_inst, d_tiles, max_polls, kp);
  return cudaGetLastError();
}

// h_inst: the host copy of the launch's only instance (constants as a kernel parameter),
// or null for launches over several instances.  max_polls: poll cap of the row waits (0: the
// full TMA_WAIT_LIMIT; a test lowers it to make a wait give up while the copies still land).
inline cudaError_t launch_tma(int thermal, int cols, const Inst* d_inst, const Tile* d_tiles, int ntiles,
                              cudaStream_t s, const Inst* h_inst, unsigned max_polls) {
  if (cols != ST_COLS) return cudaErrorInvalidValue;
  if (ntiles <= 0) return cudaSuccess;
  KParams<float> kp{};
  if (h_inst) {
    kp.I = *h_inst;
    fill_consts<float>(kp.C, *h_inst, h_inst->rho_ref);
    return thermal ? launch_tma_t<true, true>(d_inst, d_tiles, ntiles, max_polls, s, kp)
                   : launch_tma_t<false, true>(d_inst, d_tiles, ntiles, max_polls, s, kp);
  }
  return thermal ? launch_tma_t<true, false>(d_inst, d_tiles, ntiles, max_polls, s, kp)
                 : launch_tma_t<false, false>(d_inst, d_tiles, ntiles, max_polls, s, kp);
}

template <bool THERMAL>
int resident_tma_t() {
  constexpr size_t smem = tma_smem_bytes<THERMAL>();
  auto fn = lbm_tma_kernel<THERMAL, true>;
  int n = 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, ST_COLS, smem) != cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

inline int resident_tma(int thermal) { return thermal ? resident_tma_t<true>() : resident_tma_t<false>(); }

}  // namespace pplbm
