// Fused form of the coupled step: one kernel per time step, one CTA per TX x TY tile.
//
// The collide at a node needs v and T on its 1-ring (div v, grad T, lap T), v needs F on that ring,
// F needs psi on the 2-ring, psi needs rho and T there, and those need the pulled populations of the
// 2-ring. A CTA therefore works in three shared-memory stages:
//   1. tile + 2 ring: pull-stream + closures, moments rho, j, T and psi (the EOS) -> smem;
//      the tile's own nodes keep their 18 pulled populations in registers;
//   2. tile + 1 ring: F = F_int + F_ads + F_b and v = (j + F/2)/rho -> smem (tile nodes keep F, Q);
//   3. tile: isotropic grad T, lap T, grad rho, div v, the source phi and S0, both MRT collisions,
//      store f*, g* and phi.
// HBM sees the populations read once and written once plus phi (the algorithmic 152 B/node in FP32);
// the ring re-reads of neighbouring tiles' populations are served by L2. Ghost rows beyond a
// non-periodic y edge copy the edge row (moments, psi and, through the clamped stencil, F and v).
#include <cuda.h>
#include <cudaTypedefs.h>

#include "lbpc_device.cuh"
#include "lbpc_internal.h"

namespace lbpc {

namespace {

__device__ __forceinline__ int wrap_any(int x, int n) {
  while (x < 0) x += n;  // at most a few iterations: x stays within a few tiles of [0, n)
  while (x >= n) x -= n;
  return x;
}

// Post-stream populations of an interior node (no wrap, no closure): src[a][i - e_a].
template <class S, class R>
__device__ __forceinline__ void pull_interior(const PopBuf<S>& src, const R* w, long long N, int nx, long long i,
                                              R v[9]) {
#pragma unroll
  for (int a = 0; a < 9; ++a) v[a] = pop_load<S, R>(src, N, a, i - (long long)EY(a) * nx - EX(a), w);
}

// Domain row for region row offset: wraps when y is periodic, else clamps to the edge row.
__device__ __forceinline__ int row_of(const DevParams& P, int y) {
  if (P.yper) return wrap_any(y, P.ny);
  return y < 0 ? 0 : (y >= P.ny ? P.ny - 1 : y);
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// TMA staging of an interior tile: every population plane's box of the tile plus its pull halo is
// copied to shared memory by the tensor-memory accelerator, so the pulls become shared-memory reads.
// Box: BY = TY + 6 rows from y0 - 3, BX columns from x0 - XOFF (XOFF keeps the start 16-byte aligned).
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: about a second of polling at most; false if the phase did not complete.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
  for (unsigned it = 0; it < (1u << 20); ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"(tm), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(tm), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory view of a staged tile.
template <class S> struct TmaTile {
  const unsigned char* base;  // 18 population planes (f then g), then the f and g reference planes
};

template <class S, class R, int TX, int TY>
__device__ __forceinline__ void pull_staged(const TmaTile<S>& t, int set, const R* w, int hx, int hy, R v[9]) {
  using B = TmaBox<S, TX, TY>;
  const S* pop = (const S*)(t.base + (size_t)set * 9 * B::PLANE);
  const float* ref = (const float*)(t.base + 18 * B::PLANE + (size_t)set * B::RPLANE);
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const int row = hy + 1 - EY(a), col = hx + B::XOFF - 2 - EX(a);
    const S* pa = (const S*)((const unsigned char*)pop + a * B::PLANE);
    if constexpr (B::HALF) {
      v[a] = R(__half2float(pa[row * B::BX + col])) + w[a] * R(ref[row * B::REFX + col]);
    } else {
      v[a] = R(pa[row * B::BX + col]);
    }
  }
}

template <class R, int TX, int TY> struct FusedSmem {
  R rho[TY + 4][TX + 4], T[TY + 4][TX + 4], psi[TY + 4][TX + 4], jx[TY + 4][TX + 4], jy[TY + 4][TX + 4];
  R vx[TY + 2][TX + 2], vy[TY + 2][TX + 2];
  double red[TX * TY / 32];
};

// INTERIOR: the tile, its 2-ring and their pull sources lie inside the domain away from every edge,
// so no index wraps, no boundary closure applies and no ghost row exists (a per-CTA, uniform choice).
template <int MODE, class S, class R, int TX, int TY>
__device__ __forceinline__ void fused_body(const PopBuf<S>& fsrc, const PopBuf<S>& gsrc, const PopBuf<S>& fdst,
                                           const PopBuf<S>& gdst, R* __restrict__ phi_prev,
                                           const DevParams& P, long long step, int first,
                                           const double* __restrict__ rho_ave, double* __restrict__ partials,
                                           long long* __restrict__ status, FusedSmem<R, TX, TY>& sm, int x0, int y0,
                                           int pslot, const TmaTile<S> staged = TmaTile<S>{nullptr}) {
  constexpr bool INTERIOR = MODE != 0;
  constexpr int RX = TX + 4, RY = TY + 4;  // stage-1 region (tile + 2)
  constexpr int VX = TX + 2, VY = TY + 2;  // stage-2 region (tile + 1)
  (void)RY;
  constexpr int NT = TX * TY;
  auto& s_rho = sm.rho;
  auto& s_T = sm.T;
  auto& s_psi = sm.psi;
  auto& s_jx = sm.jx;
  auto& s_jy = sm.jy;
  auto& s_vx = sm.vx;
  auto& s_vy = sm.vy;
  double* s_red = sm.red;

  const Coefs<R>& C = coefs<R>(P);
  const int t = threadIdx.x;
  const int tx = t % TX, ty = t / TX;
  const int gx = x0 + tx, gy = y0 + ty;
  const bool active = gx < P.nx && gy < P.ny;
  const int mx = wrap_any(gx, P.nx), my = row_of(P, gy);

  // ---- stage 1a: own node (kept in registers) ----
  R f[9], g[9];
  if (MODE == 2) {
    pull_staged<S, R, TX, TY>(staged, 0, C.wf, tx + 2, ty + 2, f);
    pull_staged<S, R, TX, TY>(staged, 1, C.wg, tx + 2, ty + 2, g);
  } else if (INTERIOR) {
    const long long io = (long long)gy * P.nx + gx;
    pull_interior<S, R>(fsrc, C.wf, P.N, P.nx, io, f);
    pull_interior<S, R>(gsrc, C.wg, P.N, P.nx, io, g);
  } else {
    pull_closed<S, R>(fsrc, gsrc, P, mx, my, f, g);
  }
  R rho, T, p, dpdT;
  {
    rho = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
    const R jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
    const R jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
    T = g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + g[6] + g[7] + g[8];
    eos(rho, T, P, p, dpdT);
    const R psi2 = C.psi_scale * (p - rho * R(1.0 / 3.0));
    if (active) {
      const int bad = classify(rho, T, psi2, P);
      if (bad) report(status, step, gx, gy, bad);
    }
    s_rho[ty + 2][tx + 2] = rho;
    s_T[ty + 2][tx + 2] = T;
    s_psi[ty + 2][tx + 2] = sqrt(fmax(psi2, R(0)));
    s_jx[ty + 2][tx + 2] = jx;
    s_jy[ty + 2][tx + 2] = jy;
  }
  // ---- stage 1b: the 2-wide ring around the tile ----
  constexpr int RING1 = RX * RY - NT;
  for (int r = t; r < RING1; r += NT) {
    int hx, hy;
    if (r < 2 * RX) {                       // two rows below
      hx = r % RX; hy = r / RX;
    } else if (r < 4 * RX) {                // two rows above
      hx = (r - 2 * RX) % RX; hy = TY + 2 + (r - 2 * RX) / RX;
    } else {                                // two columns left and right of the tile rows
      const int q = r - 4 * RX;
      hy = 2 + q / 4;
      const int c = q % 4;
      hx = c < 2 ? c : TX + c;
    }
    R fr[9], gr[9];
    if (MODE == 2) {
      pull_staged<S, R, TX, TY>(staged, 0, C.wf, hx, hy, fr);
      pull_staged<S, R, TX, TY>(staged, 1, C.wg, hx, hy, gr);
    } else if (INTERIOR) {
      const long long io = (long long)(y0 + hy - 2) * P.nx + (x0 + hx - 2);
      pull_interior<S, R>(fsrc, C.wf, P.N, P.nx, io, fr);
      pull_interior<S, R>(gsrc, C.wg, P.N, P.nx, io, gr);
    } else {
      const int x = wrap_any(x0 + hx - 2, P.nx), y = row_of(P, y0 + hy - 2);
      pull_closed<S, R>(fsrc, gsrc, P, x, y, fr, gr);
    }
    const R rr = fr[0] + fr[1] + fr[2] + fr[3] + fr[4] + fr[5] + fr[6] + fr[7] + fr[8];
    const R Tr = gr[0] + gr[1] + gr[2] + gr[3] + gr[4] + gr[5] + gr[6] + gr[7] + gr[8];
    R pr, dr;
    eos(rr, Tr, P, pr, dr);
    const R psi2 = C.psi_scale * (pr - rr * R(1.0 / 3.0));
    s_rho[hy][hx] = rr;
    s_T[hy][hx] = Tr;
    s_psi[hy][hx] = sqrt(fmax(psi2, R(0)));
    s_jx[hy][hx] = fr[1] - fr[3] + fr[5] - fr[6] - fr[7] + fr[8];
    s_jy[hy][hx] = fr[2] - fr[4] + fr[5] + fr[6] - fr[7] - fr[8];
  }
  if (P.buoyancy) {
    const double sr = block_sum<NT>(active ? (double)rho : 0.0, s_red);
    if (t == 0) partials[pslot] = sr;
  } else {
    __syncthreads();
  }

  // ---- stage 2: F and v on tile + 1 ----
  // F at stage-2 position (vx_, vy_) of the domain node (x, y); the stencil rows come from the clamped
  // node's own region rows so a ghost position reproduces the edge node exactly.
  const R rho_ref = P.buoyancy ? R(*rho_ave) : R(0);
  auto force_at = [&](int hx, int hy, int y, R& Fx, R& Fy, R& Q, R& vx, R& vy) {
    // hx, hy: stage-1 region coordinates of the node whose F is computed
    const R c00 = s_psi[hy - 1][hx - 1], c01 = s_psi[hy - 1][hx], c02 = s_psi[hy - 1][hx + 1];
    const R c10 = s_psi[hy][hx - 1], c12 = s_psi[hy][hx + 1];
    const R c20 = s_psi[hy + 1][hx - 1], c21 = s_psi[hy + 1][hx], c22 = s_psi[hy + 1][hx + 1];
    const R pc = s_psi[hy][hx];
    const R sx = (c12 - c10) * R(1.0 / 3.0) + (c22 - c20 - c00 + c02) * R(1.0 / 12.0);
    const R sy = (c21 - c01) * R(1.0 / 3.0) + (c22 + c20 - c00 - c02) * R(1.0 / 12.0);
    Fx = -C.G * pc * sx;
    Fy = -C.G * pc * sy;
    if (!INTERIOR && !P.yper) {
      if (y == 0 && P.ybc_lo == BC_WALL) Fy += C.G_wall * 0.5f * pc;
      if (y == P.ny - 1 && P.ybc_hi == BC_WALL) Fy -= C.G_wall * 0.5f * pc;
    }
    const R rr = s_rho[hy][hx];
    if (P.buoyancy) {
      const R d = rr - rho_ref;
      Fx += d * C.gx;
      Fy += d * C.gy;
    }
    Q = C.qG2 * (sx * sx + sy * sy);
    const R ir = R(1) / rr;
    vx = (s_jx[hy][hx] + Fx * 0.5f) * ir;
    vy = (s_jy[hy][hx] + Fy * 0.5f) * ir;
  };
  // region row (stage-1 coordinates) holding the clamped domain row of stage-1 row hy
  auto clamp_hy = [&](int hy) {
    if (INTERIOR || P.yper) return hy;
    const int y = y0 + hy - 2;
    if (y < 0) return hy - y;                 // row of y = 0
    if (y >= P.ny) return hy - (y - (P.ny - 1));  // row of y = ny - 1
    return hy;
  };
  R Fx, Fy, Q, vx, vy;
  {
    const int hy = clamp_hy(ty + 2);
    force_at(tx + 2, hy, my, Fx, Fy, Q, vx, vy);
    s_vx[ty + 1][tx + 1] = vx;
    s_vy[ty + 1][tx + 1] = vy;
  }
  constexpr int RING2 = VX * VY - NT;
  for (int r = t; r < RING2; r += NT) {
    int hx, hy;  // stage-2 coordinates
    if (r < VX) {
      hx = r; hy = 0;
    } else if (r < 2 * VX) {
      hx = r - VX; hy = TY + 1;
    } else {
      const int q = r - 2 * VX;
      hy = 1 + q / 2;
      hx = (q % 2) ? TX + 1 : 0;
    }
    const int y1 = clamp_hy(hy + 1);
    const int ydom = row_of(P, y0 + hy - 1);
    R a, b, c, vxr, vyr;
    force_at(hx + 1, y1, ydom, a, b, c, vxr, vyr);
    s_vx[hy][hx] = vxr;
    s_vy[hy][hx] = vyr;
  }
  __syncthreads();

  // ---- stage 3: gradients, source, collisions on the tile ----
  if (!active) return;
  const int hx = tx + 2, hy = ty + 2;  // stage-1 coordinates of the own node
  const R gTx = (s_T[hy][hx + 1] - s_T[hy][hx - 1]) * R(1.0 / 3.0) +
                (s_T[hy + 1][hx + 1] - s_T[hy + 1][hx - 1] - s_T[hy - 1][hx - 1] + s_T[hy - 1][hx + 1]) * R(1.0 / 12.0);
  const R gTy = (s_T[hy + 1][hx] - s_T[hy - 1][hx]) * R(1.0 / 3.0) +
                (s_T[hy + 1][hx + 1] + s_T[hy + 1][hx - 1] - s_T[hy - 1][hx - 1] - s_T[hy - 1][hx + 1]) * R(1.0 / 12.0);
  const R lapT = (s_T[hy][hx + 1] + s_T[hy][hx - 1] + s_T[hy + 1][hx] + s_T[hy - 1][hx] - T * 4) * R(2.0 / 3.0) +
                 (s_T[hy + 1][hx + 1] + s_T[hy + 1][hx - 1] + s_T[hy - 1][hx - 1] + s_T[hy - 1][hx + 1] - T * 4) *
                     R(1.0 / 6.0);
  const int ux = tx + 1, uy = ty + 1;  // stage-2 coordinates
  const R divv = (s_vx[uy][ux + 1] - s_vx[uy][ux - 1]) * R(1.0 / 3.0) +
                 (s_vx[uy + 1][ux + 1] - s_vx[uy + 1][ux - 1] - s_vx[uy - 1][ux - 1] + s_vx[uy - 1][ux + 1]) * R(1.0 / 12.0) +
                 (s_vy[uy + 1][ux] - s_vy[uy - 1][ux]) * R(1.0 / 3.0) +
                 (s_vy[uy + 1][ux + 1] + s_vy[uy + 1][ux - 1] - s_vy[uy - 1][ux - 1] - s_vy[uy - 1][ux + 1]) * R(1.0 / 12.0);
  const R rcv = rho * C.cV;
  const R inv_rcv = R(1) / rcv;
  R div_lam_gradT;
  if (P.lambda_mode == 0) {
    div_lam_gradT = C.lambda * lapT;
  } else {
    const R grx = (s_rho[hy][hx + 1] - s_rho[hy][hx - 1]) * R(1.0 / 3.0) +
                  (s_rho[hy + 1][hx + 1] - s_rho[hy + 1][hx - 1] - s_rho[hy - 1][hx - 1] + s_rho[hy - 1][hx + 1]) * R(1.0 / 12.0);
    const R gry = (s_rho[hy + 1][hx] - s_rho[hy - 1][hx]) * R(1.0 / 3.0) +
                  (s_rho[hy + 1][hx + 1] + s_rho[hy + 1][hx - 1] - s_rho[hy - 1][hx - 1] - s_rho[hy - 1][hx + 1]) * R(1.0 / 12.0);
    div_lam_gradT = rcv * C.chi * lapT + C.cV_chi * (grx * gTx + gry * gTy);
  }
  const long long i = (long long)gy * P.nx + gx;
  const R compress = T * (R(1) - dpdT * inv_rcv) * divv;
  R phi, S0, tau_inv = R(0);
  if (P.model == 2) {  // Gong-Cheng: Eq. 13 source, local tau_g (Sec. IV A)
    phi = compress;
    S0 = phi;
    tau_inv = R(1) / ((P.lambda_mode == 0 ? C.lambda * 3 * inv_rcv : C.chi * 3) + R(0.5));
  } else {
    phi = div_lam_gradT * inv_rcv - C.kdiff * lapT + compress;
    S0 = phi;
    if (P.model == 0) {
      const R pp = first ? phi : phi_prev[i];
      S0 = phi + (phi - pp) * 0.5f;
    }
  }
  phi_prev[i] = phi;
  collide_flow(f, rho, vx, vy, Fx, Fy, Q, P);
  collide_heat(g, T, vx, vy, S0, P, tau_inv);
  pop_store<S, R>(fdst, P.N, i, f, rho, C.wf);
  pop_store<S, R>(gdst, P.N, i, g, T + S0, C.wg);
}

template <class S, class R, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) k_fused(PopBuf<S> fsrc, PopBuf<S> gsrc, PopBuf<S> fdst, PopBuf<S> gdst,
                                                   R* __restrict__ phi_prev, DevParams P, long long step, int first,
                                                   const double* __restrict__ rho_ave, double* __restrict__ partials,
                                                   long long* __restrict__ status) {
  __shared__ FusedSmem<R, TX, TY> sm;
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const bool interior = x0 >= 3 && x0 + TX + 3 <= P.nx && y0 >= 3 && y0 + TY + 3 <= P.ny;
  const int pslot = blockIdx.y * gridDim.x + blockIdx.x;
  if (interior)
    fused_body<1, S, R, TX, TY>(fsrc, gsrc, fdst, gdst, phi_prev, P, step, first, rho_ave, partials, status, sm, x0, y0,
                                pslot);
  else
    fused_body<0, S, R, TX, TY>(fsrc, gsrc, fdst, gdst, phi_prev, P, step, first, rho_ave, partials, status, sm, x0, y0,
                                pslot);
}

// Same step with the interior tiles' populations staged in shared memory by TMA (dynamic shared
// memory of TmaBox<S, TX, TY>::BYTES). Tiles that touch an edge take the general path.
template <class S, class R, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) k_fused_tma(PopBuf<S> fsrc, PopBuf<S> gsrc, PopBuf<S> fdst, PopBuf<S> gdst,
                                                       R* __restrict__ phi_prev, DevParams P, long long step, int first,
                                                       const double* __restrict__ rho_ave,
                                                       double* __restrict__ partials, long long* __restrict__ status,
                                                       const __grid_constant__ TmaMaps maps) {
  using B = TmaBox<S, TX, TY>;
  __shared__ FusedSmem<R, TX, TY> sm;
  extern __shared__ __align__(128) unsigned char dyn[];
  const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
  const bool interior = x0 >= 3 && x0 + TX + 3 <= P.nx && y0 >= 3 && y0 + TY + 3 <= P.ny;
  const int pslot = blockIdx.y * gridDim.x + blockIdx.x;
  if (!interior) {
    fused_body<0, S, R, TX, TY>(fsrc, gsrc, fdst, gdst, phi_prev, P, step, first, rho_ave, partials, status, sm, x0, y0,
                                pslot);
    return;
  }
  uint64_t* bar = (uint64_t*)(dyn + B::BYTES - 128);
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_expect_tx(bar, (unsigned)(18 * B::BX * B::BY * sizeof(S) + (B::HALF ? 2 * B::REFX * B::BY * 4 : 0)));
    for (int a = 0; a < 9; ++a) {
      tma_load_3d(dyn + a * B::PLANE, &maps.f, x0 - B::XOFF, y0 - 3, a, bar);
      tma_load_3d(dyn + (9 + a) * B::PLANE, &maps.g, x0 - B::XOFF, y0 - 3, a, bar);
    }
    if (B::HALF) {
      tma_load_2d(dyn + 18 * B::PLANE, &maps.rf, x0 - B::XOFF, y0 - 3, bar);
      tma_load_2d(dyn + 18 * B::PLANE + B::RPLANE, &maps.rg, x0 - B::XOFF, y0 - 3, bar);
    }
  }
  if (!mbar_wait_bounded(bar, 0)) {
    if (threadIdx.x == 0) report(status, step, x0, y0, ST_TIMEOUT);
    mbar_wait_bounded(bar, 0);  // let the copies in flight land before the block's shared memory goes away
    return;
  }
  fused_body<2, S, R, TX, TY>(fsrc, gsrc, fdst, gdst, phi_prev, P, step, first, rho_ave, partials, status, sm, x0, y0,
                              pslot, TmaTile<S>{dyn});
}

// ------------------------------------------------------------------------------------------------
template <class S, class R, int TX, int TY>
static cudaError_t fused_impl(const SplitBuffers& b, const DevParams& P, int cur, long long step, cudaStream_t st,
                              cudaEvent_t* ev) {
  dim3 grid((P.nx + TX - 1) / TX, (P.ny + TY - 1) / TY);
  const PopBuf<S> fs{(S*)b.f[cur], b.ref_f[cur]}, gs{(S*)b.g[cur], b.ref_g[cur]};
  const PopBuf<S> fd{(S*)b.f[cur ^ 1], b.ref_f[cur ^ 1]}, gd{(S*)b.g[cur ^ 1], b.ref_g[cur ^ 1]};
  if (ev) cudaEventRecord(ev[0], st);
  bool staged = false;
  if constexpr (sizeof(S) <= 4) {  // the TMA-staged kernel exists for FP32 and FP16 storage
    if (b.tma[cur]) {
      using B = TmaBox<S, TX, TY>;
      static bool attr = false;
      if (!attr) {
        cudaFuncSetAttribute(k_fused_tma<S, R, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, B::BYTES);
        attr = true;
      }
      k_fused_tma<S, R, TX, TY><<<grid, TX * TY, B::BYTES, st>>>(fs, gs, fd, gd, (R*)b.phi_prev, P, step, step == 0,
                                                                 b.scalars, b.partials, b.status, *b.tma[cur]);
      staged = true;
    }
  }
  if (!staged)
    k_fused<S, R, TX, TY><<<grid, TX * TY, 0, st>>>(fs, gs, fd, gd, (R*)b.phi_prev, P, step, step == 0, b.scalars,
                                                    b.partials, b.status);
  if (ev) cudaEventRecord(ev[1], st);
  if (P.buoyancy) {
    fused_finish(b, P, (int)(grid.x * grid.y), st);
    if (ev) cudaEventRecord(ev[2], st);
  }
  return cudaGetLastError();
}

// ---- tensor maps of the TMA-staged path ----
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

template <class S, int TX, int TY>
static bool encode_t(TmaMaps* m, void* f, void* g, float* rf, float* rg, const DevParams& P) {
  using B = TmaBox<S, TX, TY>;
  auto fn = encode_fn();
  if (!fn) return false;
  if (((size_t)P.nx * sizeof(S)) % 16 != 0) return false;  // row stride must be a multiple of 16 bytes
  const CUtensorMapDataType dt = sizeof(S) == 2 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                : (sizeof(S) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64);
  const cuuint64_t dims[3] = {(cuuint64_t)P.nx, (cuuint64_t)P.ny, 9};
  const cuuint64_t strides[2] = {(cuuint64_t)P.nx * sizeof(S), (cuuint64_t)P.N * sizeof(S)};
  const cuuint32_t box[3] = {(cuuint32_t)B::BX, (cuuint32_t)B::BY, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  auto enc3 = [&](CUtensorMap* t, void* base) {
    return fn(t, dt, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  };
  if (!enc3(&m->f, f) || !enc3(&m->g, g)) return false;
  if (B::HALF) {
    const cuuint64_t d2[2] = {(cuuint64_t)P.nx, (cuuint64_t)P.ny};
    const cuuint64_t s2[1] = {(cuuint64_t)P.nx * 4};
    const cuuint32_t b2[2] = {(cuuint32_t)B::REFX, (cuuint32_t)B::BY};
    auto enc2 = [&](CUtensorMap* t, void* base) {
      return fn(t, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, d2, s2, b2, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
             CUDA_SUCCESS;
    };
    if (!enc2(&m->rf, rf) || !enc2(&m->rg, rg)) return false;
  }
  return true;
}

bool fused_tma_encode(TmaMaps* m, int prec, int tile, void* f, void* g, float* rf, float* rg, const DevParams& P) {
  if (prec == 1) return tile ? encode_t<float, 32, 8>(m, f, g, rf, rg, P) : encode_t<float, 32, 16>(m, f, g, rf, rg, P);
  if (prec == 2)
    return tile ? encode_t<__half, 32, 8>(m, f, g, rf, rg, P) : encode_t<__half, 32, 16>(m, f, g, rf, rg, P);
  return false;  // FP64 runs the split step by default; its fused form keeps per-thread loads
}

cudaError_t fused_step(const SplitBuffers& b, const DevParams& P, int prec, int cur, long long step, cudaStream_t st,
                       cudaEvent_t* ev) {
  if (prec == 0) {
    SplitBuffers nb = b;
    nb.tma[0] = nb.tma[1] = nullptr;
    return fused_impl<double, double, 32, 8>(nb, P, cur, step, st, ev);
  }
  if (prec == 3) {
    SplitBuffers nb = b;
    nb.tma[0] = nb.tma[1] = nullptr;
    return fused_impl<dw, dw, 32, 8>(nb, P, cur, step, st, ev);
  }
  if (prec == 1)
    return b.fused_tile ? fused_impl<float, float, 32, 8>(b, P, cur, step, st, ev)
                        : fused_impl<float, float, 32, 16>(b, P, cur, step, st, ev);
  return b.fused_tile ? fused_impl<__half, float, 32, 8>(b, P, cur, step, st, ev)
                      : fused_impl<__half, float, 32, 16>(b, P, cur, step, st, ev);
}

// ------------------------------------------------------------------------------------------------
// Batched step: many independent instances of uneven size in one persistent launch. CTAs walk a work
// list of (instance, tile) entries round-robin (the tiles in flight at any moment form one compact
// band of the list, so neighbouring tiles' halos meet in L2); each tile runs the same body as the
// single-instance kernel with that instance's parameters and buffers, so an instance's result does
// not depend on what else is in the batch. The tile count and every per-instance value live in
// device memory, so a captured CUDA graph of these launches stays valid when instances join or leave.
//
// The walk is software-pipelined: while a tile computes, the CTA already holds the next tile's list
// entry and copies the next instance's descriptor (integer header, the coefficient set of the
// arithmetic type, buffer pointers and step state) into the second of two shared-memory slots with
// 16-byte asynchronous copies, so a change of instance costs no exposed global-memory latency.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

template <class R> struct CoefSpan;  // byte range of the coefficient set a kernel of arithmetic R reads
template <> struct CoefSpan<double> { static constexpr size_t off = offsetof(DevParams, cd), len = sizeof(Coefs<double>); };
template <> struct CoefSpan<float> { static constexpr size_t off = offsetof(DevParams, cf), len = sizeof(Coefs<float>); };
template <> struct CoefSpan<dw> { static constexpr size_t off = offsetof(DevParams, cw), len = sizeof(Coefs<dw>); };

// Copy the parts of an instance descriptor a kernel of arithmetic R reads, in 16-byte chunks issued by
// the first threads of the block; completes at the issuing threads' next cp_async_wait_all.
template <class S, class R>
__device__ __forceinline__ void desc_copy_async(BatchInst<S>* dst, const BatchInst<S>* src) {
  constexpr size_t HEAD = offsetof(DevParams, cd) / 16;                 // nx .. heat_unit_rates
  constexpr size_t COEF = (CoefSpan<R>::len + 15) / 16;                  // the coefficient set
  constexpr size_t TAIL_OFF = offsetof(BatchInst<S>, f);                 // pointers and step state
  constexpr size_t TAIL = (sizeof(BatchInst<S>) - TAIL_OFF) / 16;
  static_assert(offsetof(DevParams, cd) % 16 == 0 && CoefSpan<R>::off % 16 == 0 && TAIL_OFF % 16 == 0 &&
                    sizeof(BatchInst<S>) % 16 == 0,
                "descriptor parts must be 16-byte aligned");
  static_assert(CoefSpan<R>::off + 16 * COEF <= sizeof(DevParams), "coefficient span inside the parameters");
  const unsigned char* s = (const unsigned char*)src;
  unsigned char* d = (unsigned char*)dst;
  const int k = threadIdx.x;
  if (k < (int)HEAD) {
    cp_async16(d + 16 * k, s + 16 * k);
  } else if (k < (int)(HEAD + COEF)) {
    const size_t o = CoefSpan<R>::off + 16 * (k - HEAD);
    cp_async16(d + o, s + o);
  } else if (k < (int)(HEAD + COEF + TAIL)) {
    const size_t o = TAIL_OFF + 16 * (k - HEAD - COEF);
    cp_async16(d + o, s + o);
  }
}

template <class S, class R, int TX, int TY>
__global__ void __launch_bounds__(TX* TY, sizeof(S) <= 4 ? 1024 / (TX * TY) : 1)
    k_batch_step(const BatchMeta* __restrict__ meta, const BatchInst<S>* __restrict__ insts) {
  static_assert(TX * TY >= 128, "the descriptor copy needs at least 128 threads");
  static_assert(sizeof(BatchTile) == 16, "a work-list entry is one 16-byte copy");
  __shared__ FusedSmem<R, TX, TY> sm;
  __shared__ BatchInst<S> sI[2];
  __shared__ BatchTile st[3];  // this tile's entry, the next one's, and the one after (filled while computing)
  const int ntiles = meta->ntiles;
  const BatchTile* __restrict__ tiles = meta->tiles;
  const int G = gridDim.x;
  int t = blockIdx.x;
  if (t >= ntiles) return;
  if (threadIdx.x == 0) {
    st[0] = tiles[t];
    if (t + G < ntiles) st[1] = tiles[t + G];
  }
  __syncthreads();
  desc_copy_async<S, R>(&sI[0], &insts[st[0].inst]);
  cp_async_wait_all();
  __syncthreads();
  int slot = 0, r = 0;  // descriptor slot of this tile; ring position of this tile's entry
  for (;;) {
    const BatchTile tile = st[r];
    const int rn = r == 2 ? 0 : r + 1, ra = rn == 2 ? 0 : rn + 1;
    const bool more = t + G < ntiles;
    const bool change = more && st[rn].inst != tile.inst;
    if (change) desc_copy_async<S, R>(&sI[slot ^ 1], &insts[st[rn].inst]);
    if (threadIdx.x == TX * TY - 1 && t + 2 * G < ntiles) cp_async16(&st[ra], &tiles[t + 2 * G]);
    const BatchInst<S>& I = sI[slot];
    const DevParams& P = I.P;
    const int cur = I.cur;
    const long long step = I.step;
    const bool interior = tile.x0 >= 3 && tile.x0 + TX + 3 <= P.nx && tile.y0 >= 3 && tile.y0 + TY + 3 <= P.ny;
    if (interior)
      fused_body<1, S, R, TX, TY>(I.f[cur], I.g[cur], I.f[cur ^ 1], I.g[cur ^ 1], (R*)I.phi_prev, P, step, step == 0,
                                  I.scalars, I.partials, I.status, sm, tile.x0, tile.y0, tile.pslot);
    else
      fused_body<0, S, R, TX, TY>(I.f[cur], I.g[cur], I.f[cur ^ 1], I.g[cur ^ 1], (R*)I.phi_prev, P, step, step == 0,
                                  I.scalars, I.partials, I.status, sm, tile.x0, tile.y0, tile.pslot);
    cp_async_wait_all();
    __syncthreads();  // the tile is done with the shared memory; the next descriptor and entry have landed
    if (!more) break;
    if (change) slot ^= 1;
    t += G;
    r = rn;
  }
}

// One block per instance slot: rho_ave from the tile partials (fixed order), then flip the buffers
// and count the step.
template <class S>
__global__ void __launch_bounds__(128) k_batch_advance(BatchInst<S>* __restrict__ insts) {
  __shared__ double red[4];
  BatchInst<S>& I = insts[blockIdx.x];
  if (!I.active) return;
  if (I.P.buoyancy) {
    double acc = 0.0;
    for (int j = threadIdx.x; j < I.ntiles; j += 128) acc += I.partials[j];
    acc = block_sum<128>(acc, red);
    if (threadIdx.x == 0) I.scalars[0] = acc / (double)I.P.N;
  }
  if (threadIdx.x == 0) {
    I.cur ^= 1;
    I.step += 1;
  }
}

template <class S, class R, int TX, int TY>
static cudaError_t batch_launch_t(int ctas, const BatchMeta* d_meta, void* d_insts, int ninst, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_batch_step<S, R, TX, TY><<<sms * ctas, TX * TY, 0, st>>>(d_meta, (const BatchInst<S>*)d_insts);
  if (ninst > 0) k_batch_advance<S><<<ninst, 128, 0, st>>>((BatchInst<S>*)d_insts);
  return cudaGetLastError();
}

template <class S, class R>
static cudaError_t batch_launch_p(int variant, int ctas, const BatchMeta* d_meta, void* d_insts, int ninst,
                                  cudaStream_t st) {
  if (variant == 1) return batch_launch_t<S, R, 32, 16>(ctas, d_meta, d_insts, ninst, st);
  if (variant == 2) return batch_launch_t<S, R, 64, 8>(ctas, d_meta, d_insts, ninst, st);
  return batch_launch_t<S, R, 32, 8>(ctas, d_meta, d_insts, ninst, st);
}

cudaError_t batch_step_launch(int prec, int variant, int ctas, const BatchMeta* d_meta, void* d_insts, int ninst,
                              cudaStream_t st) {
  if (prec == 0) return batch_launch_p<double, double>(variant, ctas, d_meta, d_insts, ninst, st);
  if (prec == 1) return batch_launch_p<float, float>(variant, ctas, d_meta, d_insts, ninst, st);
  return batch_launch_p<__half, float>(variant, ctas, d_meta, d_insts, ninst, st);
}

template <class S, class R, int TX, int TY> static int occ_t() {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_step<S, R, TX, TY>, TX * TY, 0);
  return n;
}

template <class S, class R> static int occ_p(int variant) {
  if (variant == 1) return occ_t<S, R, 32, 16>();
  if (variant == 2) return occ_t<S, R, 64, 8>();
  return occ_t<S, R, 32, 8>();
}

int batch_max_ctas_per_sm(int prec, int variant) {
  if (prec == 0) return occ_p<double, double>(variant);
  if (prec == 1) return occ_p<float, float>(variant);
  return occ_p<__half, float>(variant);
}

}  // namespace lbpc
