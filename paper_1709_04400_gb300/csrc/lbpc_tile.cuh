// The tile body of the fused and batched steps: one CTA per TX x TY tile of a domain.
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
#pragma once

#include <cuda.h>
#include <stddef.h>

#include <type_traits>

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
template <class S, class R, class IX = long long>
__device__ __forceinline__ void pull_interior(const PopBuf<S>& src, const R* w, IX N, int nx, IX i, R v[9]) {
#pragma unroll
  for (int a = 0; a < 9; ++a) v[a] = pop_load<S, R, IX>(src, N, a, i - (IX)EY(a) * nx - EX(a), w);
}

// Domain row for region row offset: wraps when y is periodic, else clamps to the edge row.
template <class PT> __device__ __forceinline__ int row_of(const PT& P, int y) {
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

// Resident CTAs per SM requested of the compiler for the tile kernels with 4- and 2-byte storage:
// 1024 threads per SM with one node per thread (64 registers), 512 with two (128 registers, which
// the two nodes' populations need). 8-byte storage is left unconstrained.
template <class S, int NTH, int NPT> __host__ __device__ constexpr int fused_min_blocks() {
  return sizeof(S) <= 4 ? ((NPT == 1 ? 1024 : 512) / NTH > 0 ? (NPT == 1 ? 1024 : 512) / NTH : 1) : 1;
}

// INTERIOR: the tile, its 2-ring and their pull sources lie inside the domain away from every edge,
// so no index wraps, no boundary closure applies and no ghost row exists (a per-CTA, uniform choice).
// NPT nodes per thread: a CTA of TX * TY / NPT threads; thread t owns tile nodes t + k * (TX * TY / NPT),
// k < NPT, and keeps their populations in registers from stage 1 to stage 3. With NPT = 2 the ring
// stages keep more of the (fewer) threads busy and every thread carries two independent chains.
// IDX32: population indices formed in 32 bits (the caller guarantees 9 N < 2^31), and loads and stores
// issued as global ones explicitly. This is for buffers whose pointers come from a descriptor in shared
// memory (the batch's work-list kernel): the compiler cannot infer their space, and each wider index costs
// registers there. Where the pointers and sizes are kernel parameters, 64-bit indices are faster.
// after_stage1: called by every thread once the tile has finished reading its staged populations (after
// the block barrier that closes stage 1); the persistent TMA kernel starts the next tile's copy there.
struct NoStageHook {
  __device__ __forceinline__ void operator()() const {}
};

template <int MODE, class S, class R, int TX, int TY, int NPT = 1, bool IDX32 = false, class PT = DevParams,
          class AfterStage1 = NoStageHook>
__device__ __forceinline__ void fused_body(const PopBuf<S>& fsrc, const PopBuf<S>& gsrc, const PopBuf<S>& fdst,
                                           const PopBuf<S>& gdst, R* __restrict__ phi_prev,
                                           const PT& P, long long step, int first,
                                           const double* __restrict__ rho_ave, double* __restrict__ partials,
                                           long long* __restrict__ status, FusedSmem<R, TX, TY>& sm, int x0, int y0,
                                           int pslot, const TmaTile<S> staged = TmaTile<S>{nullptr},
                                           const long long* step_at = nullptr,
                                           AfterStage1 after_stage1 = AfterStage1{}) {
  constexpr bool INTERIOR = MODE != 0;
  using IX = typename std::conditional<IDX32, int, long long>::type;
  constexpr int RX = TX + 4, RY = TY + 4;  // stage-1 region (tile + 2)
  constexpr int VX = TX + 2, VY = TY + 2;  // stage-2 region (tile + 1)
  (void)RY;
  constexpr int NN = TX * TY;              // tile nodes
  constexpr int NTH = NN / NPT;            // threads
  static_assert(NN % NPT == 0 && NTH % 32 == 0, "whole warps");
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

  // ---- stage 1a: own nodes (kept in registers) ----
  R f[NPT][9], g[NPT][9];
  R rho[NPT], T[NPT], dpdT[NPT];
  R pp[NPT];  // phi of the previous step, loaded here so that the load overlaps stages 1-2
  int my[NPT];
  bool active[NPT];
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int n = t + k * NTH;
    const int tx = n % TX, ty = n / TX;
    const int gx = x0 + tx, gy = y0 + ty;
    active[k] = gx < P.nx && gy < P.ny;
    if constexpr (IDX32)
      pp[k] = (active[k] && P.model == 0 && !first) ? __ldg(phi_prev + ((IX)gy * P.nx + gx)) : R(0);
    else
      pp[k] = (active[k] && P.model == 0 && !first) ? phi_prev[(long long)gy * P.nx + gx] : R(0);
    const int mx = wrap_any(gx, P.nx);
    my[k] = row_of(P, gy);
    if (MODE == 2) {
      pull_staged<S, R, TX, TY>(staged, 0, C.wf, tx + 2, ty + 2, f[k]);
      pull_staged<S, R, TX, TY>(staged, 1, C.wg, tx + 2, ty + 2, g[k]);
    } else if (INTERIOR) {
      const IX io = (IX)gy * P.nx + gx;
      pull_interior<S, R, IX>(fsrc, C.wf, (IX)P.N, P.nx, io, f[k]);
      pull_interior<S, R, IX>(gsrc, C.wg, (IX)P.N, P.nx, io, g[k]);
    } else {
      pull_closed<S, R, IX>(fsrc, gsrc, P, mx, my[k], f[k], g[k]);
    }
    const R* fk = f[k];
    const R* gk = g[k];
    rho[k] = density_of(fk);
    const R jx = fk[1] - fk[3] + fk[5] - fk[6] - fk[7] + fk[8];
    const R jy = fk[2] - fk[4] + fk[5] + fk[6] - fk[7] - fk[8];
    R Tlo;
    T[k] = heat_of(gk, Tlo);
    R p;
    eos(rho[k], T[k], P, p, dpdT[k]);
    const R psi2 = psi_squared(p, dpdT[k], Tlo, rho[k], C);
    if (active[k]) {
      const int bad = classify(rho[k], T[k], psi2, P);
      if (bad) report(status, step_at ? *step_at : step, gx, gy, bad);  // step_at: read only to report
    }
    s_rho[ty + 2][tx + 2] = rho[k];
    s_T[ty + 2][tx + 2] = T[k];
    s_psi[ty + 2][tx + 2] = sqrt(fmax(psi2, R(0)));
    s_jx[ty + 2][tx + 2] = jx;
    s_jy[ty + 2][tx + 2] = jy;
  }
  // ---- stage 1b: the 2-wide ring around the tile ----
  constexpr int RING1 = RX * RY - NN;
  for (int r = t; r < RING1; r += NTH) {
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
      const IX io = (IX)(y0 + hy - 2) * P.nx + (x0 + hx - 2);
      pull_interior<S, R, IX>(fsrc, C.wf, (IX)P.N, P.nx, io, fr);
      pull_interior<S, R, IX>(gsrc, C.wg, (IX)P.N, P.nx, io, gr);
    } else {
      const int x = wrap_any(x0 + hx - 2, P.nx), y = row_of(P, y0 + hy - 2);
      pull_closed<S, R, IX>(fsrc, gsrc, P, x, y, fr, gr);
    }
    const R rr = density_of(fr);
    R Trlo;
    const R Tr = heat_of(gr, Trlo);
    R pr, dr;
    eos(rr, Tr, P, pr, dr);
    const R psi2 = psi_squared(pr, dr, Trlo, rr, C);
    s_rho[hy][hx] = rr;
    s_T[hy][hx] = Tr;
    s_psi[hy][hx] = sqrt(fmax(psi2, R(0)));
    s_jx[hy][hx] = fr[1] - fr[3] + fr[5] - fr[6] - fr[7] + fr[8];
    s_jy[hy][hx] = fr[2] - fr[4] + fr[5] + fr[6] - fr[7] - fr[8];
  }
  if (P.buoyancy == 1) {
    double own = 0.0;
#pragma unroll
    for (int k = 0; k < NPT; ++k) own += active[k] ? (double)rho[k] : 0.0;
    const double sr = block_sum<NTH>(own, s_red);
    if (t == 0) partials[pslot] = sr;
  } else {
    __syncthreads();
  }
  after_stage1();

  // ---- stage 2: F and v on tile + 1 ----
  // F at stage-2 position (vx_, vy_) of the domain node (x, y); the stencil rows come from the clamped
  // node's own region rows so a ghost position reproduces the edge node exactly.
  const R rho_ref = P.buoyancy == 1 ? R(*rho_ave) : (P.buoyancy == 2 ? C.rho_bc_hi : R(0));
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
    // F_ads = -G_w psi(x) sum_a w_a psi(x) s(x+e_a) e_a, on the y- wall only (a y+ wall is a neutral lid)
    if (!INTERIOR && !P.yper && y == 0 && P.ybc_lo == BC_WALL) Fy += C.G_wall * 0.5f * pc * pc;
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
  R Fx[NPT], Fy[NPT], Q[NPT], vx[NPT], vy[NPT];
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int n = t + k * NTH;
    const int tx = n % TX, ty = n / TX;
    const int hy = clamp_hy(ty + 2);
    force_at(tx + 2, hy, my[k], Fx[k], Fy[k], Q[k], vx[k], vy[k]);
    s_vx[ty + 1][tx + 1] = vx[k];
    s_vy[ty + 1][tx + 1] = vy[k];
  }
  constexpr int RING2 = VX * VY - NN;
  for (int r = t; r < RING2; r += NTH) {
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
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    if (!active[k]) continue;
    const int n = t + k * NTH;
    const int tx = n % TX, ty = n / TX;
    const int gx = x0 + tx, gy = y0 + ty;
    const int hx = tx + 2, hy = ty + 2;  // stage-1 coordinates of the own node
    const R Tk = T[k];
    const R gTx = (s_T[hy][hx + 1] - s_T[hy][hx - 1]) * R(1.0 / 3.0) +
                  (s_T[hy + 1][hx + 1] - s_T[hy + 1][hx - 1] - s_T[hy - 1][hx - 1] + s_T[hy - 1][hx + 1]) * R(1.0 / 12.0);
    const R gTy = (s_T[hy + 1][hx] - s_T[hy - 1][hx]) * R(1.0 / 3.0) +
                  (s_T[hy + 1][hx + 1] + s_T[hy + 1][hx - 1] - s_T[hy - 1][hx - 1] - s_T[hy - 1][hx + 1]) * R(1.0 / 12.0);
    const R lapT = (s_T[hy][hx + 1] + s_T[hy][hx - 1] + s_T[hy + 1][hx] + s_T[hy - 1][hx] - Tk * 4) * R(2.0 / 3.0) +
                   (s_T[hy + 1][hx + 1] + s_T[hy + 1][hx - 1] + s_T[hy - 1][hx - 1] + s_T[hy - 1][hx + 1] - Tk * 4) *
                       R(1.0 / 6.0);
    const int ux = tx + 1, uy = ty + 1;  // stage-2 coordinates
    const R divv = (s_vx[uy][ux + 1] - s_vx[uy][ux - 1]) * R(1.0 / 3.0) +
                   (s_vx[uy + 1][ux + 1] - s_vx[uy + 1][ux - 1] - s_vx[uy - 1][ux - 1] + s_vx[uy - 1][ux + 1]) * R(1.0 / 12.0) +
                   (s_vy[uy + 1][ux] - s_vy[uy - 1][ux]) * R(1.0 / 3.0) +
                   (s_vy[uy + 1][ux + 1] + s_vy[uy + 1][ux - 1] - s_vy[uy - 1][ux - 1] - s_vy[uy - 1][ux + 1]) * R(1.0 / 12.0);
    const R rcv = rho[k] * C.cV;
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
    const IX i = (IX)gy * P.nx + gx;
    const R compress = Tk * (R(1) - dpdT[k] * inv_rcv) * divv;
    R phi, S0, tau_inv = R(0);
    if (P.model == 2) {  // Gong-Cheng: Eq. 13 source, local tau_g (Sec. IV A)
      phi = compress;
      S0 = phi;
      tau_inv = R(1) / ((P.lambda_mode == 0 ? C.lambda * 3 * inv_rcv : C.chi * 3) + R(0.5));
    } else {
      phi = div_lam_gradT * inv_rcv - C.kdiff * lapT + compress;
      S0 = phi;
      if (P.model == 0) S0 = phi + (phi - (first ? phi : pp[k])) * 0.5f;
    }
    if constexpr (IDX32)
      __stwb(phi_prev + i, phi);
    else
      phi_prev[i] = phi;
    collide_flow(f[k], rho[k], vx[k], vy[k], Fx[k], Fy[k], Q[k], P);
    collide_heat(g[k], Tk, vx[k], vy[k], S0, P, tau_inv);
    if constexpr (IDX32) {
      pop_store_global<S, R, IX>(fdst, (IX)P.N, i, f[k], rho[k], C.wf);
      pop_store_global<S, R, IX>(gdst, (IX)P.N, i, g[k], Tk + S0, C.wg);
    } else {
      pop_store<S, R>(fdst, P.N, i, f[k], rho[k], C.wf);
      pop_store<S, R>(gdst, P.N, i, g[k], Tk + S0, C.wg);
    }
    if (!INTERIOR) wall_force_store(fdst.wall, P, gx, gy, Fx[k], Fy[k]);
  }
}

}  // namespace lbpc
