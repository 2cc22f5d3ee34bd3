// Device-side building blocks of the coupled step: D2Q9 lattice, Peng-Robinson EOS, boundary
// closures, moment transforms and the two MRT collisions. Every kernel of liblbpc composes these,
// so that the split and fused kernels compute the same arithmetic.
//
// D2Q9 order: e0=(0,0) e1=(1,0) e2=(0,1) e3=(-1,0) e4=(0,-1) e5=(1,1) e6=(-1,1) e7=(-1,-1) e8=(1,-1);
// weights 4/9, 1/9, 1/36 (Sec. II B). Moments (rho, e, eps, jx, qx, jy, qy, pxx, pxy): the orthogonal
// MRT basis of Eqs. 42-43, whose thermal equilibria are Eq. 53.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#include "lbpc_dw.cuh"

namespace lbpc {

enum { BC_PERIODIC = 0, BC_WALL = 1, BC_PRESSURE = 2 };
enum { ST_RHO_LE0 = 1, ST_RHO_POLE = 2, ST_T_LE0 = 3, ST_PSI2_NEG = 4, ST_NONFINITE = 5, ST_TIMEOUT = 6 };

__host__ __device__ constexpr int EX(int a) { return a == 1 || a == 5 || a == 8 ? 1 : (a == 3 || a == 6 || a == 7 ? -1 : 0); }
__host__ __device__ constexpr int EY(int a) { return a == 2 || a == 5 || a == 6 ? 1 : (a == 4 || a == 7 || a == 8 ? -1 : 0); }

// Real-valued parameters in the arithmetic type of a kernel, folded on the host, so that a kernel
// never converts between FP64 and FP32 (on GB300 those conversions run at the FP64 rate).
template <class R> struct Coefs {
  R T_bc[4], T_strip;
  R rho_bc_lo, rho_bc_hi;
  R a, b, R_gas, G, kappa;
  R s_f[9], s_g[9];
  R lambda, chi, cV, kdiff;  // kdiff = (1/s_g3 - 1/2) c_s^2
  R gx, gy, G_wall;
  R c3, c5;     // (1 - s3/2) s4, (1 - s5/2) s6 of Eqs. 54-55
  R inv_Tc;     // 1 / T_c
  R hf[9];      // 1 - s_f[k]/2, the forcing weights of (I - Lambda/2) S_F
  R qG2;        // 12 sigma / (1/s_e - 1/2) * G^2: Q = qcoef |F_int|^2 / psi^2 = qG2 |sum_a w psi e|^2
  R inv_cV;     // 1 / c_V
  R psi_scale;  // 2 / G: psi^2 = (2/G) (p - rho c_s^2)
  R cV_chi;     // c_V chi
  R wf[9];      // rest-state equilibrium weights of f: M^{-1} m_eq(1, v = 0) = (4/9, 1/9 x4, 1/36 x4)
  R wg[9];      // rest-state equilibrium weights of g: M^{-1} m_eq(T = 1, v = 0) of the thermal model
};

// Everything a kernel needs, derived once on the host from lbpc_params and passed by value. The
// coefficient sets start on 16-byte boundaries so that a kernel can copy the header and the one set
// it uses with 16-byte asynchronous copies.
struct alignas(16) DevParams {
  int nx, ny;
  long long N;       // nx * ny
  int yper;          // y periodic
  int ybc_lo, ybc_hi;
  int tbc[4];
  int strip_x0, strip_x1;
  int model;         // 0 improved, 1 compromised
  int lambda_mode;   // 0 const, 1 rho cV chi
  int buoyancy;
  int heat_unit_rates;  // s_g[1..8] all 1: the thermal relaxation sets every non-conserved moment to m_eq
  alignas(16) Coefs<double> cd;
  alignas(16) Coefs<float> cf;
  alignas(16) Coefs<dw> cw;  // double-word arithmetic (LBPC_DF64)
};

template <class R> __host__ __device__ __forceinline__ const Coefs<R>& coefs(const DevParams& P);
template <> __host__ __device__ __forceinline__ const Coefs<double>& coefs<double>(const DevParams& P) { return P.cd; }
template <> __host__ __device__ __forceinline__ const Coefs<float>& coefs<float>(const DevParams& P) { return P.cf; }
template <> __host__ __device__ __forceinline__ const Coefs<dw>& coefs<dw>(const DevParams& P) { return P.cw; }

// The header of DevParams with the one coefficient set of arithmetic R: what a kernel of that arithmetic
// reads, in a third of the bytes, for parameters that are copied per launch (the batch's per-tile
// launches). The device helpers take either form (template parameter PT).
template <class R> struct alignas(16) DevParamsOf {
  int nx, ny;
  long long N;
  int yper;
  int ybc_lo, ybc_hi;
  int tbc[4];
  int strip_x0, strip_x1;
  int model;
  int lambda_mode;
  int buoyancy;
  int heat_unit_rates;
  alignas(16) Coefs<R> c;
};
static_assert(offsetof(DevParamsOf<float>, c) == offsetof(DevParams, cd) &&
                  offsetof(DevParamsOf<float>, heat_unit_rates) == offsetof(DevParams, heat_unit_rates),
              "DevParamsOf repeats the header of DevParams");
template <class R> __host__ __device__ __forceinline__ const Coefs<R>& coefs(const DevParamsOf<R>& P) { return P.c; }
template <class R> inline DevParamsOf<R> params_of(const DevParams& P) {
  DevParamsOf<R> q;
  memcpy(&q, &P, offsetof(DevParams, cd));  // the common header
  q.c = coefs<R>(P);
  return q;
}

// ------------------------------------------------------------------------------------------------
// moment transforms: m = M x and x = M^{-1} m with M^{-1} = M^T diag(1/9,1/36,1/36,1/6,1/12,1/6,1/12,1/4,1/4)
// ------------------------------------------------------------------------------------------------
template <class R> __device__ __forceinline__ void to_moments(const R x[9], R m[9]) {
  const R s14 = x[1] + x[2] + x[3] + x[4];
  const R s58 = x[5] + x[6] + x[7] + x[8];
  const R d13 = x[1] - x[3], d24 = x[2] - x[4];
  const R px = x[5] - x[6] - x[7] + x[8];
  const R py = x[5] + x[6] - x[7] - x[8];
  m[0] = x[0] + s14 + s58;
  m[1] = x[0] * -4 - s14 + s58 * 2;
  m[2] = x[0] * 4 - s14 * 2 + s58;
  m[3] = d13 + px;
  m[4] = d13 * -2 + px;
  m[5] = d24 + py;
  m[6] = d24 * -2 + py;
  m[7] = x[1] - x[2] + x[3] - x[4];
  m[8] = x[5] - x[6] + x[7] - x[8];
}

template <class R> __device__ __forceinline__ void from_moments(const R m[9], R x[9]) {
  const R u0 = m[0] * R(1.0 / 9.0), u1 = m[1] * R(1.0 / 36.0), u2 = m[2] * R(1.0 / 36.0);
  const R u3 = m[3] * R(1.0 / 6.0), u4 = m[4] * R(1.0 / 12.0), u5 = m[5] * R(1.0 / 6.0);
  const R u6 = m[6] * R(1.0 / 12.0), u7 = m[7] * R(0.25), u8 = m[8] * R(0.25);
  const R ax = u0 - u1 - u2 * 2;  // common to e1..e4
  const R dg = u0 + u1 * 2 + u2;  // common to e5..e8
  const R qx = u3 - u4 * 2, qy = u5 - u6 * 2;
  const R sx = u3 + u4, sy = u5 + u6;
  x[0] = u0 - u1 * 4 + u2 * 4;
  x[1] = ax + qx + u7;
  x[2] = ax + qy - u7;
  x[3] = ax - qx + u7;
  x[4] = ax - qy - u7;
  x[5] = dg + sx + sy + u8;
  x[6] = dg - sx + sy - u8;
  x[7] = dg - sx - sy + u8;
  x[8] = dg + sx - sy - u8;
}

// x = M^{-1} m for the post-collision populations. In binary32 arithmetic the rest population is taken
// as x0 = m0 - (x1 + ... + x8), so that the populations sum to the zeroth moment up to one rounding:
// the scale 1/9 of m0 rounds up by 7.5e-9 in binary32, and the plain transform would scale each node's
// mass (or heat) by 9 fl(1/9) in every collision, a steady drift of about 1e-8 per step. In binary64
// and double-word arithmetic that drift is about 5e-17 per step, and the plain transform is kept (the
// double-word type's lazy additions lose accuracy in the longer sum).
template <class R> __device__ __forceinline__ void from_moments_conserving(const R m[9], R x[9]) {
  from_moments(m, x);
  if constexpr (sizeof(R) == 4) x[0] = m[0] - (((x[1] + x[2]) + (x[3] + x[4])) + ((x[5] + x[6]) + (x[7] + x[8])));
}

// ------------------------------------------------------------------------------------------------
// Peng-Robinson EOS (Eq. 56) and (dp/dT)_rho
// ------------------------------------------------------------------------------------------------
template <class R, class PT> __device__ __forceinline__ void eos(R rho, R T, const PT& P, R& p, R& dpdT, R* inv_rho = nullptr) {
  const Coefs<R>& C = coefs<R>(P);
  // theta(T) = [1 + kappa (1 - sqrt(T/T_c))]^2 and d theta/dT = -kappa [..] / sqrt(T T_c); one rsqrt
  // gives both sqrt(T/T_c) = t rsqrt(t) and 1/sqrt(T T_c) = rsqrt(t) / T_c with t = T/T_c.
  const R t = T * C.inv_Tc;
  const R rs = rsqrt(t);
  const R sq = t * rs;
  const R th1 = R(1) + C.kappa * (R(1) - sq);
  const R theta = th1 * th1;
  const R dtheta = -C.kappa * th1 * rs * C.inv_Tc;
  // 1/(1 - b rho) and 1/(1 + 2 b rho - b^2 rho^2) (and 1/rho if asked) from one reciprocal
  const R br = C.b * rho;
  const R d1 = R(1) - br;
  const R d2 = R(1) + br * 2 - br * br;
  const R d12 = d1 * d2;
  R r12;
  if (inv_rho) {
    const R r = R(1) / (rho * d12);
    *inv_rho = d12 * r;
    r12 = rho * r;
  } else {
    r12 = R(1) / d12;
  }
  const R inv1 = d2 * r12, inv2 = d1 * r12;
  const R r2 = rho * rho;
  p = rho * C.R_gas * T * inv1 - C.a * theta * r2 * inv2;
  dpdT = rho * C.R_gas * inv1 - C.a * dtheta * r2 * inv2;
}

// ------------------------------------------------------------------------------------------------
// zeroth moments and the pseudopotential in binary32
// ------------------------------------------------------------------------------------------------
// In binary32 a plain sum of nine populations rounds up to eight times at the scale of the result.
// Near rest the populations stand in fixed ratios to the rest population (D2Q9 flow weights: f_a = f0/4
// on the axes, 4 f_a = f0/4 on the diagonals; thermal weights of the improved model, g0 = 5T/9 and
// g_a = T/18 = g0/10, within a factor 2 of g0/8), and a difference of two binary32 numbers within a
// factor 2 of each other is exact (Sterbenz). The sums below take every population relative to that ratio first, so
// the large part is one exact product of the rest population and the rounding falls on small
// deviations. Binary64 and double-word arithmetic keep the plain sums.
template <class R> __device__ __forceinline__ R density_of(const R f[9]) {
  if constexpr (sizeof(R) == 4) {
    const R q = f[0] * 0.25f;
    const R A = ((f[1] - q) + (f[2] - q)) + ((f[3] - q) + (f[4] - q));
    const R B = (fmaf(4.f, f[5], -q) + fmaf(4.f, f[6], -q)) + (fmaf(4.f, f[7], -q) + fmaf(4.f, f[8], -q));
    return fmaf(2.25f, f[0], A + B * 0.25f);  // rho = 9 f0/4 + A + B/4
  } else {
    return f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
  }
}

// Temperature T = sum g. In binary32 also its rounding residual lo (T + lo is the sum of the deviations
// to within their own small roundings): the liquid's pressure changes with T about 30 times faster than
// with rho in lattice units, so the residual is carried into psi^2 (psi_squared).
template <class R> __device__ __forceinline__ R heat_of(const R g[9], R& lo) {
  if constexpr (sizeof(R) == 4) {
    const R q = g[0] * 0.125f;
    const R E = (((g[1] - q) + (g[2] - q)) + ((g[3] - q) + (g[4] - q))) +
                (((g[5] - q) + (g[6] - q)) + ((g[7] - q) + (g[8] - q)));
    const R t2 = g[0] * 2.f;
    const R T = t2 + E;  // T = 2 g0 + sum (g_a - g0/8)
    lo = E - (T - t2);   // exact residual (Fast2Sum: |2 g0| > |E|)
    return T;
  } else {
    lo = R(0);
    return g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + g[6] + g[7] + g[8];
  }
}

// psi^2 = (2/G)(p_EOS - rho c_s^2) (reading of Ref. [48]), with p_EOS first moved by (dp/dT)_rho Tlo
// for the residual of a binary32 temperature (zero otherwise).
template <class R>
__device__ __forceinline__ R psi_squared(R p, R dpdT, R Tlo, R rho, const Coefs<R>& C) {
  if constexpr (sizeof(R) == 4) return C.psi_scale * ((p + dpdT * Tlo) - rho * R(1.0 / 3.0));
  else return C.psi_scale * (p - rho * R(1.0 / 3.0));
}

// ------------------------------------------------------------------------------------------------
// population storage
// ------------------------------------------------------------------------------------------------
// One population set (f or g) in one buffer: SoA [9][N] of the storage type S. With S = __half the
// stored value is the deviation of the post-collision population from the rest-state equilibrium
// w_a * ref of the node that stored it, ref being that node's density (f) or post-collision
// temperature (g), held in an FP32 plane beside the populations. The collision conserves the zeroth
// moment, so the deviations are of order |u| w rho and keep binary16's 11 bits relative to them.
//
// A flow buffer also carries the force on its wall rows (`wall`, FP64 [edge y-/y+][Fx/Fy][nx]), written
// by the step that stored the populations: the next step's wall closure sets j = -F/2 from it.
template <class S> struct PopBuf {
  S* p;
  float* ref;    // FP16 storage only
  double* wall;  // flow buffers: wall-row forces (null where unused; aggregate init leaves it null)
};

// Index of a wall row's entries in PopBuf::wall: edge 0 = y-, 1 = y+; component 0 = Fx, 1 = Fy.
__host__ __device__ __forceinline__ long long wall_slot(int nx, int edge, int comp, int x) {
  return (long long)(2 * edge + comp) * nx + x;
}
// doubles of one wall-force buffer (one parity)
__host__ __device__ __forceinline__ long long wall_doubles(int nx) { return 4LL * nx; }

template <class S> struct is_half_t { static constexpr bool value = false; };
template <> struct is_half_t<__half> { static constexpr bool value = true; };

// IX is the index type: long long in general; int where the caller guarantees that every population
// index of the buffer (9 N) fits in 31 bits, which turns each address into one 32-bit multiply-add.
template <class S, class R, class IX = long long>
__device__ __forceinline__ R pop_load(const PopBuf<S>& b, IX N, int a, IX idx, const R* w) {
  if constexpr (is_half_t<S>::value) {
    return R(__half2float(__ldg(b.p + ((IX)a * N + idx)))) + w[a] * R(__ldg(b.ref + idx));
  } else if constexpr (is_dw_t<S>::value) {
    return R(ldgv(b.p + ((IX)a * N + idx)));
  } else {
    return R(__ldg(b.p + ((IX)a * N + idx)));
  }
}

// Store the post-collision populations v of node i; refval is the node's zeroth moment after the
// collision (rho for f, T + S0 for g), the reference of the FP16 deviation.
template <class S, class R, class IX = long long>
__device__ __forceinline__ void pop_store(const PopBuf<S>& b, IX N, IX i, const R v[9], R refval, const R* w) {
  if constexpr (is_half_t<S>::value) {
#pragma unroll
    for (int a = 0; a < 9; ++a) b.p[(IX)a * N + i] = __float2half_rn(float(v[a] - w[a] * refval));
    b.ref[i] = float(refval);
  } else {
#pragma unroll
    for (int a = 0; a < 9; ++a) b.p[(IX)a * N + i] = (S)v[a];
  }
}

// pop_store through explicitly global stores, for buffer pointers that the compiler cannot place in
// the global space (descriptors read from shared memory).
template <class S, class R, class IX = long long>
__device__ __forceinline__ void pop_store_global(const PopBuf<S>& b, IX N, IX i, const R v[9], R refval,
                                                 const R* w) {
  if constexpr (is_half_t<S>::value) {
#pragma unroll
    for (int a = 0; a < 9; ++a) __stwb(b.p + ((IX)a * N + i), __float2half_rn(float(v[a] - w[a] * refval)));
    __stwb(b.ref + i, float(refval));
  } else {
#pragma unroll
    for (int a = 0; a < 9; ++a) __stwb(b.p + ((IX)a * N + i), (S)v[a]);
  }
}

// ------------------------------------------------------------------------------------------------
// pull-stream with the boundary closures applied at the pulling node
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ int wrapx(int x, int nx) { return x < 0 ? x + nx : (x >= nx ? x - nx : x); }

// Post-stream populations at (x, y): src holds post-collision populations (SoA [9][N]); a
// population whose source node lies beyond a non-periodic y edge is unknown and returned as 0.
//
// The nine source nodes (x - e_a) share three columns and three rows; PullSrc holds them once per node
// (x, y inside the grid), wrapped on the periodic axes. Entry k of each array is the source for e = k - 1.
struct PullSrc {
  int col[3];  // x + 1, x, x - 1 (wrapped)
  int row[3];  // y + 1, y, y - 1 (wrapped when y is periodic; -1 beyond a non-periodic y edge)
};
template <class PT> __device__ __forceinline__ PullSrc pull_src(const PT& P, int x, int y) {
  PullSrc s;
  s.col[0] = x == P.nx - 1 ? 0 : x + 1;
  s.col[1] = x;
  s.col[2] = x == 0 ? P.nx - 1 : x - 1;
  s.row[0] = y == P.ny - 1 ? (P.yper ? 0 : -1) : y + 1;
  s.row[1] = y;
  s.row[2] = y == 0 ? (P.yper ? P.ny - 1 : -1) : y - 1;
  return s;
}

template <class S, class R, class IX = long long, class PT = DevParams>
__device__ __forceinline__ void pull_from(const PopBuf<S>& src, const R* w, const PT& P, const PullSrc& s,
                                          R v[9]) {
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    const int r = s.row[EY(a) + 1];
    v[a] = r >= 0 ? pop_load<S, R, IX>(src, (IX)P.N, a, (IX)r * P.nx + s.col[EX(a) + 1], w) : R(0);
  }
}

template <class S, class R, class PT>
__device__ __forceinline__ void pull(const PopBuf<S>& src, const R* w, const PT& P, int x, int y, R v[9]) {
  pull_from<S, R>(src, w, P, pull_src(P, x, y), v);
}

// Zou-He closure of the unknown f on a non-periodic y edge. Wall: the momentum is set to j = -F/2, F
// being the wall row's force of the step that stored the populations (`wall`, see PopBuf), so that the
// forcing scheme's velocity v = (j + F/2)/rho vanishes on the wall (a null `wall` reads as F = 0).
// Pressure: rho = rho_bc, u_x = 0.
template <class R, class PT>
__device__ __forceinline__ void flow_closure(R f[9], const PT& P, int x, int y, const double* wall) {
  if (P.yper) return;
  const Coefs<R>& C = coefs<R>(P);
  const R d13 = f[1] - f[3];
  if (y == 0) {
    if (P.ybc_lo == BC_WALL) {  // f2 - f4 = 2/3 j_y; f5 - f6 closes j_x
      const R jx = wall ? R(wall[wall_slot(P.nx, 0, 0, x)]) * -0.5f : R(0);
      const R jy = wall ? R(wall[wall_slot(P.nx, 0, 1, x)]) * -0.5f : R(0);
      f[2] = f[4] + R(2.0 / 3.0) * jy;
      f[5] = f[7] - d13 * 0.5f + jx * 0.5f + jy * R(1.0 / 6.0);
      f[6] = f[8] + d13 * 0.5f - jx * 0.5f + jy * R(1.0 / 6.0);
    } else {
      const R ru = C.rho_bc_lo - (f[0] + f[1] + f[3] + (f[4] + f[7] + f[8]) * 2);  // rho_bc u_y
      f[2] = f[4] + R(2.0 / 3.0) * ru;
      f[5] = f[7] - d13 * 0.5f + ru * R(1.0 / 6.0);
      f[6] = f[8] + d13 * 0.5f + ru * R(1.0 / 6.0);
    }
  } else if (y == P.ny - 1) {
    if (P.ybc_hi == BC_WALL) {
      const R jx = wall ? R(wall[wall_slot(P.nx, 1, 0, x)]) * -0.5f : R(0);
      const R jy = wall ? R(wall[wall_slot(P.nx, 1, 1, x)]) * -0.5f : R(0);
      f[4] = f[2] - R(2.0 / 3.0) * jy;
      f[7] = f[5] + d13 * 0.5f - jx * 0.5f - jy * R(1.0 / 6.0);
      f[8] = f[6] - d13 * 0.5f + jx * 0.5f - jy * R(1.0 / 6.0);
    } else {
      const R ru = (f[0] + f[1] + f[3] + (f[2] + f[5] + f[6]) * 2) - C.rho_bc_hi;  // rho_bc u_y
      f[4] = f[2] - R(2.0 / 3.0) * ru;
      f[7] = f[5] + d13 * 0.5f - ru * R(1.0 / 6.0);
      f[8] = f[6] - d13 * 0.5f - ru * R(1.0 / 6.0);
    }
  }
}

// Thermal equilibrium moments (Eq. 53 for the improved model, Eq. 44 for the compromised one, and for
// the Gong-Cheng model the moments of Eq. 14: the second-order equilibrium with rho replaced by T).
template <class R> __device__ __forceinline__ void heat_meq(R T, R vx, R vy, int model, R n[9]) {
  if (model == 2) {
    const R v2 = vx * vx + vy * vy;
    n[0] = T;
    n[1] = T * (R(-2) + v2 * 3);
    n[2] = T * (R(1) - v2 * 3);
    n[3] = T * vx;
    n[4] = -T * vx;
    n[5] = T * vy;
    n[6] = -T * vy;
    n[7] = T * (vx * vx - vy * vy);
    n[8] = T * vx * vy;
    return;
  }
  n[0] = T;
  n[1] = T * -2;
  n[2] = model == 0 ? T * 2 : T;
  n[3] = T * vx;
  n[4] = -T * vx;
  n[5] = T * vy;
  n[6] = -T * vy;
  n[7] = R(0);
  n[8] = R(0);
}

// Thermal boundary step. On a non-periodic y edge the unknown g are closed by bounce-back:
// g_a = -g_opp(a) + 2 g_a^eq(T_bc, 0) where the edge holds T_bc (anti-bounce-back; heat enters through
// the wall), g_a = g_opp(a) otherwise (zero heat flux). A Dirichlet edge of a periodic axis (a ring
// inside a periodic domain) resets the node to g := M^{-1} m_eq(T_bc, 0): x edges, then y edges.
template <class R, class PT> __device__ __forceinline__ void heat_closure(R g[9], const PT& P, int x, int y) {
  const Coefs<R>& C = coefs<R>(P);
  if (!P.yper) {
    if (y == 0) {
      if (P.tbc[2]) {
        const R Tb = (x >= P.strip_x0 && x < P.strip_x1) ? C.T_strip : C.T_bc[2];
        R n[9], e[9];
        heat_meq(Tb, R(0), R(0), P.model, n);
        from_moments(n, e);
        g[2] = e[2] * 2 - g[4];
        g[5] = e[5] * 2 - g[7];
        g[6] = e[6] * 2 - g[8];
      } else {
        g[2] = g[4]; g[5] = g[7]; g[6] = g[8];
      }
    }
    if (y == P.ny - 1) {
      if (P.tbc[3]) {
        R n[9], e[9];
        heat_meq(C.T_bc[3], R(0), R(0), P.model, n);
        from_moments(n, e);
        g[4] = e[4] * 2 - g[2];
        g[7] = e[7] * 2 - g[5];
        g[8] = e[8] * 2 - g[6];
      } else {
        g[4] = g[2]; g[7] = g[5]; g[8] = g[6];
      }
    }
  }
  bool set = false;
  R Tb = R(0);
  if (x == 0 && P.tbc[0]) { set = true; Tb = C.T_bc[0]; }
  if (x == P.nx - 1 && P.tbc[1]) { set = true; Tb = C.T_bc[1]; }
  if (P.yper) {
    if (y == 0 && P.tbc[2]) { set = true; Tb = (x >= P.strip_x0 && x < P.strip_x1) ? C.T_strip : C.T_bc[2]; }
    if (y == P.ny - 1 && P.tbc[3]) { set = true; Tb = C.T_bc[3]; }
  }
  if (set) {
    R n[9];
    heat_meq(Tb, R(0), R(0), P.model, n);
    from_moments(n, g);
  }
}

// Post-stream, post-boundary f and g at (x, y).
template <class S, class R, class IX = long long, class PT = DevParams>
__device__ __forceinline__ void pull_closed(const PopBuf<S>& fsrc, const PopBuf<S>& gsrc, const PT& P, int x,
                                            int y, R f[9], R g[9]) {
  const Coefs<R>& C = coefs<R>(P);
  const PullSrc src = pull_src(P, x, y);  // f and g read the same nine source nodes
  pull_from<S, R, IX>(fsrc, C.wf, P, src, f);
  pull_from<S, R, IX>(gsrc, C.wg, P, src, g);
  flow_closure(f, P, x, y, fsrc.wall);
  heat_closure(g, P, x, y);
}

// Keep the force of a wall-row node for the next step's closure (into the destination flow buffer).
template <class R, class PT>
__device__ __forceinline__ void wall_force_store(double* wall, const PT& P, int x, int y, R Fx, R Fy) {
  if (P.yper || !wall) return;
  const int edge = (y == 0 && P.ybc_lo == BC_WALL) ? 0 : (y == P.ny - 1 && P.ybc_hi == BC_WALL) ? 1 : -1;
  if (edge < 0) return;
  wall[wall_slot(P.nx, edge, 0, x)] = double(Fx);
  wall[wall_slot(P.nx, edge, 1, x)] = double(Fy);
}

// ------------------------------------------------------------------------------------------------
// collisions
// ------------------------------------------------------------------------------------------------
// Flow MRT collision with forcing (reading of the improved pseudopotential model, Refs. [13,29]):
// m* = m - Lambda (m - m_eq) + (I - Lambda/2) S_F, S_F with the sigma term Q in the energy moments.
//
// Binary32 takes the collision in increments, f* = f + M^{-1} (m* - m), so that every stored population
// is rounded once at its own scale. Rebuilding f* from all nine post-collision moments rounds several
// times at the scale of the populations, and the roundings of the opposite pair e_a, -e_a differ, which
// moves momentum at random. The non-equilibrium parts m - m_eq of the energy and stress moments come
// from the populations' exact deviations from their rest-state ratios (see density_of), not from moments
// of size about 2 rho that cancel. Binary64 and double-word arithmetic rebuild f* from m*.
template <class R, class PT>
__device__ __forceinline__ void collide_flow(R f[9], R rho, R vx, R vy, R Fx, R Fy, R Q, const PT& P) {
  const Coefs<R>& C = coefs<R>(P);
  const R vxx = vx * vx, vyy = vy * vy;
  const R v2 = vxx + vyy;
  const R vF = vx * Fx + vy * Fy;
  if constexpr (sizeof(R) == 4) {
    const R q = f[0] * 0.25f;
    const R d1 = f[1] - q, d2 = f[2] - q, d3 = f[3] - q, d4 = f[4] - q;
    const R d5 = fmaf(4.f, f[5], -q), d6 = fmaf(4.f, f[6], -q), d7 = fmaf(4.f, f[7], -q), d8 = fmaf(4.f, f[8], -q);
    const R A = (d1 + d2) + (d3 + d4), B = (d5 + d6) + (d7 + d8);
    const R e_dev = A + B;                       // m1 + 2 rho
    const R eps_dev = A * -3.f;                  // m2 - rho
    const R pxx = (d1 + d3) - (d2 + d4);         // m7
    const R pxy = ((d5 + d7) - (d6 + d8)) * 0.25f;  // m8
    const R qx = (f[1] - f[3]) * -2.f + ((f[5] - f[6]) + (f[8] - f[7]));  // m4
    const R qy = (f[2] - f[4]) * -2.f + ((f[5] - f[7]) + (f[6] - f[8]));  // m6
    const R r3v2 = rho * v2 * 3.f;
    R dm[9], df[9];
    dm[0] = R(0);  // S_F,0 = 0 and m0_eq = rho
    dm[3] = Fx;    // j* = j + F whatever s_j (m_eq,3 = j + F/2)
    dm[5] = Fy;
    dm[1] = C.hf[1] * (vF * 6 + Q) - C.s_f[1] * (e_dev - r3v2);  // m1 - m1_eq = (m1 + 2 rho) - 3 rho v^2
    dm[2] = C.hf[2] * (vF * -6 - Q) - C.s_f[2] * (eps_dev + r3v2);  // m2 - m2_eq = (m2 - rho) + 3 rho v^2
    dm[4] = C.hf[4] * -Fx - C.s_f[4] * (qx + rho * vx);
    dm[6] = C.hf[6] * -Fy - C.s_f[6] * (qy + rho * vy);
    dm[7] = C.hf[7] * ((vx * Fx - vy * Fy) * 2) - C.s_f[7] * (pxx - rho * (vxx - vyy));
    dm[8] = C.hf[8] * (vx * Fy + vy * Fx) - C.s_f[8] * (pxy - rho * vx * vy);
    from_moments(dm, df);
#pragma unroll
    for (int a = 0; a < 9; ++a) f[a] = f[a] + df[a];
    return;
  }
  R m[9];
  to_moments(f, m);
  // conserved moments: m0* = m0 = rho (S_F,0 = 0, m0_eq = rho; rho is the caller's sum of these f) and
  // j* = j + F whatever s_j (m_eq,3 = j + F/2)
  m[0] = rho;
  m[3] += Fx;
  m[5] += Fy;
  R meq[9], SF[9];
  meq[1] = rho * (R(-2) + v2 * 3); SF[1] = vF * 6 + Q;
  meq[2] = rho * (R(1) - v2 * 3);  SF[2] = vF * -6 - Q;
  meq[4] = -rho * vx;                 SF[4] = -Fx;
  meq[6] = -rho * vy;                 SF[6] = -Fy;
  meq[7] = rho * (vxx - vyy);         SF[7] = (vx * Fx - vy * Fy) * 2;
  meq[8] = rho * vx * vy;             SF[8] = vx * Fy + vy * Fx;
#pragma unroll
  for (int k = 1; k < 9; ++k) {
    if (k == 3 || k == 5) continue;
    m[k] = m[k] - C.s_f[k] * (m[k] - meq[k]) + C.hf[k] * SF[k];
  }
  from_moments_conserving(m, f);
}

// Thermal MRT collision of the improved model: Eq. 45 with m_eq of Eq. 53 and S = (S0, 0, ..., 0)
// (Eq. 46), then m3* += (1 - s3/2) s4 (m4 - m4_eq) and m5* += (1 - s5/2) s6 (m6 - m6_eq) (Eqs. 54-55).
template <class R, class PT>
__device__ __forceinline__ void collide_heat(R g[9], R T, R vx, R vy, R S0, const PT& P, R tau_inv = R(0)) {
  const Coefs<R>& C = coefs<R>(P);
  R ns[9];
  if (P.model == 2) {
    // Gong-Cheng (Eqs. 12-14): BGK with the local 1/tau_g, source G_a = w_a phi, whose moments are
    // phi (1, -2, 1, 0, ..., 0)
    R n[9], neq[9];
    to_moments(g, n);
    heat_meq(T, vx, vy, 2, neq);
#pragma unroll
    for (int k = 0; k < 9; ++k) ns[k] = n[k] - tau_inv * (n[k] - neq[k]);
    ns[0] += S0;
    ns[1] += S0 * -2;
    ns[2] += S0;
  } else if (P.heat_unit_rates && P.model == 0) {
    // s_k = 1 for k >= 1 (so c3 = c5 = 1/2): every non-conserved moment takes its Eq. 53 value and
    // n* = (T + S0, -2T, 2T, T vx + (n4 + T vx)/2, -T vx, T vy + (n6 + T vy)/2, -T vy, 0, 0). Its
    // back-transform M^{-1} n* in closed form: the axes and the diagonals share the base
    // B = (T + S0)/9 - T/18, the axes add +-X (+-Y) with X = 5 T vx/12 + n4/12, the diagonals +-X' +-Y'
    // with X' = T vx/6 + n4/12, and the rest population is B + T/2.
    const R TS = T + S0;
    const R Tvx = T * vx, Tvy = T * vy;
    const R n4 = (g[1] - g[3]) * -2 + (g[5] - g[6] - g[7] + g[8]);
    const R n6 = (g[2] - g[4]) * -2 + (g[5] + g[6] - g[7] - g[8]);
    const R h4 = n4 * R(1.0 / 12.0), h6 = n6 * R(1.0 / 12.0);
    const R X = Tvx * R(5.0 / 12.0) + h4, Xd = Tvx * R(1.0 / 6.0) + h4;
    const R Y = Tvy * R(5.0 / 12.0) + h6, Yd = Tvy * R(1.0 / 6.0) + h6;
    const R B = TS * R(1.0 / 9.0) - T * R(1.0 / 18.0);
    const R P1 = B + Xd, P2 = B - Xd;
    g[1] = B + X;
    g[3] = B - X;
    g[2] = B + Y;
    g[4] = B - Y;
    g[5] = P1 + Yd;
    g[8] = P1 - Yd;
    g[6] = P2 + Yd;
    g[7] = P2 - Yd;
    // binary32 keeps the heat of the node to one rounding (see from_moments_conserving)
    if constexpr (sizeof(R) == 4) g[0] = TS - (((g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8])));
    else g[0] = B + T * 0.5f;
    return;
  } else if (P.heat_unit_rates) {
    // compromised model with s_k = 1 for k >= 1: every non-conserved moment relaxes to its equilibrium,
    // so only the zeroth moment (T) is needed.
    heat_meq(T, vx, vy, P.model, ns);  // Eq. 44: n7 = n8 = 0
    ns[0] = T + S0;
  } else {
    R n[9], neq[9];
    to_moments(g, n);
    heat_meq(T, vx, vy, P.model, neq);
    ns[0] = n[0] + S0;  // n0_eq = T = n0: the relaxation leaves the zeroth moment, the source adds S0
#pragma unroll
    for (int k = 1; k < 9; ++k) ns[k] = n[k] - C.s_g[k] * (n[k] - neq[k]);
    if (P.model == 0) {
      ns[3] += C.c3 * (n[4] - neq[4]);
      ns[5] += C.c5 * (n[6] - neq[6]);
    }
  }
  from_moments_conserving(ns, g);
}

// ------------------------------------------------------------------------------------------------
// block reduction (fixed order: warp shuffle tree, then warp 0 over the warp sums)
// ------------------------------------------------------------------------------------------------
template <int BLOCK> __device__ __forceinline__ double block_sum(double v, double* smem) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) smem[w] = v;
  __syncthreads();
  double s = 0.0;
  if (w == 0) {
    s = lane < BLOCK / 32 ? smem[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  __syncthreads();
  return s;  // valid in thread 0
}

// Record the first non-physical node (step, x, y, code); later reports are dropped.
__device__ __forceinline__ void report(long long* status, long long step, int x, int y, int code) {
  if (atomicCAS((unsigned long long*)status, 0ull, 1ull) == 0ull) {
    status[1] = step;
    status[2] = x;
    status[3] = y;
    status[4] = code;
  }
}

template <class R, class PT> __device__ __forceinline__ int classify(R rho, R T, R psi2, const PT& P) {
  if constexpr (sizeof(R) == 8 && !is_dw_t<R>::value) {
    // binary64: the same tests on the bit patterns, on the integer pipe (the FP64 pipe bounds this step).
    // A finite double is positive exactly when its bits, read as a signed integer, are; b rho >= 1 for
    // a positive finite b rho exactly when its bits are at least those of 1.0; -0.0 counts as >= 0.
    const long long EXP = 0x7ff0000000000000LL;
    const long long ir = __double_as_longlong(rho), iT = __double_as_longlong(T), ip = __double_as_longlong(psi2);
    if ((ir & EXP) == EXP || (iT & EXP) == EXP || (ip & EXP) == EXP) return ST_NONFINITE;
    if (ir <= 0) return ST_RHO_LE0;
    if (__double_as_longlong(coefs<R>(P).b * rho) >= 0x3ff0000000000000LL) return ST_RHO_POLE;
    if (iT <= 0) return ST_T_LE0;
    if (ip < 0 && ip != (long long)0x8000000000000000ULL) return ST_PSI2_NEG;
    return 0;
  }
  if (!isfinite(rho) || !isfinite(T) || !isfinite(psi2)) return ST_NONFINITE;
  if (!(rho > R(0))) return ST_RHO_LE0;
  if (!(coefs<R>(P).b * rho < R(1))) return ST_RHO_POLE;
  if (!(T > R(0))) return ST_T_LE0;
  if (!(psi2 >= R(0))) return ST_PSI2_NEG;
  return 0;
}

}  // namespace lbpc
