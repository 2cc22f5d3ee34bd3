// Split form of the coupled step: three node-parallel kernels per time step.
//
//   k_macro    pull-stream + boundary closures; rho, j, T (moments), p_EOS -> psi and (dp/dT)_rho
//              (Eq. 56); optional per-block partial sums of rho for the buoyancy reference rho_ave.
//   k_force    psi stencil -> F = F_int + F_ads + F_b, v = (j + F/2)/rho, sigma term Q.
//   k_collide  pull again (same closures); isotropic grad T, lap T, grad rho, div v; source phi of
//              Eq. 28 and S0 of Eq. 46; flow MRT collide with forcing; thermal MRT collide with the
//              corrections of Eqs. 54-55; store post-collision f*, g* (pull scheme, A/B buffers).
//
// Each kernel reads its node's stencil straight from global memory (L1/L2 serve the reuse). With
// FP64 arithmetic the step is bound by the FP64 pipe, not by HBM, and this split computes every
// EOS evaluation, force and velocity exactly once per node and step.
#include "lbpc_device.cuh"
#include "lbpc_internal.h"

namespace lbpc {

constexpr int BLOCK = 64;  // small blocks spread small grids evenly over the 152 SMs

// Planes of the split path's scratch (type R, N nodes each).
enum { P_RHO = 0, P_T, P_PSI, P_JX, P_JY, P_DPDT, P_IRHO, P_VX, P_VY, P_FX, P_FY, P_Q, NPLANES };

template <class R> struct Planes {
  R* p[NPLANES];
};

__device__ __forceinline__ long long node_index(const DevParams& P, int x, int y) { return (long long)y * P.nx + x; }

// Neighbour row for a stencil: wraps when y is periodic, else clamps to the edge row (ghost rows
// copy the edge row). out_lo/out_hi report a ghost beyond the lower / upper edge.
__device__ __forceinline__ int nb_row(const DevParams& P, int y, int dy, bool& ghost_lo, bool& ghost_hi) {
  int yy = y + dy;
  ghost_lo = ghost_hi = false;
  if (P.yper) return yy < 0 ? yy + P.ny : (yy >= P.ny ? yy - P.ny : yy);
  if (yy < 0) { ghost_lo = true; return 0; }
  if (yy >= P.ny) { ghost_hi = true; return P.ny - 1; }
  return yy;
}

// Gather the 3x3 neighbourhood c[dy+1][dx+1] of a plane with the copy-ghost rule.
template <class R> __device__ __forceinline__ void gather9(const R* __restrict__ X, const DevParams& P, int x, int y, R c[3][3]) {
  const int xm = wrapx(x - 1, P.nx), xp = wrapx(x + 1, P.nx);
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy) {
    bool lo, hi;
    const long long row = (long long)nb_row(P, y, dy, lo, hi) * P.nx;
    c[dy + 1][0] = ldgv(X + row + xm);
    c[dy + 1][1] = ldgv(X + row + x);
    c[dy + 1][2] = ldgv(X + row + xp);
  }
}

// Isotropic differences (reading of the paper's cited stencils): d_i X = 3 sum_a w_a X(x+e_a) e_ai,
// lap X = 6 sum_a w_a (X(x+e_a) - X(x)). c[1][1] is the centre, c[2][*] the row above.
template <class R> __device__ __forceinline__ R d_x(const R c[3][3]) {
  return (c[1][2] - c[1][0]) * R(1.0 / 3.0) + (c[2][2] - c[2][0] - c[0][0] + c[0][2]) * R(1.0 / 12.0);
}
template <class R> __device__ __forceinline__ R d_y(const R c[3][3]) {
  return (c[2][1] - c[0][1]) * R(1.0 / 3.0) + (c[2][2] + c[2][0] - c[0][0] - c[0][2]) * R(1.0 / 12.0);
}
template <class R> __device__ __forceinline__ R lap(const R c[3][3]) {
  const R ctr = c[1][1];
  return (c[1][2] + c[1][0] + c[2][1] + c[0][1] - ctr * 4) * R(2.0 / 3.0) +
         (c[2][2] + c[2][0] + c[0][0] + c[0][2] - ctr * 4) * R(1.0 / 6.0);
}

template <class S, class R>
__global__ void __launch_bounds__(BLOCK) k_macro(PopBuf<S> fsrc, PopBuf<S> gsrc, Planes<R> pl,
                                                 DevParams P, long long step, int do_partials,
                                                 double* __restrict__ partials, long long* __restrict__ status) {
  __shared__ double red[BLOCK / 32];
  const Coefs<R>& C = coefs<R>(P);
  const long long i = (long long)blockIdx.x * BLOCK + threadIdx.x;
  double rho_d = 0.0;
  if (i < P.N) {
    const int y = (int)(i / P.nx), x = (int)(i - (long long)y * P.nx);
    R f[9], g[9];
    pull_closed<S, R>(fsrc, gsrc, P, x, y, f, g);
    const R rho = density_of(f);
    const R jx = f[1] - f[3] + f[5] - f[6] - f[7] + f[8];
    const R jy = f[2] - f[4] + f[5] + f[6] - f[7] - f[8];
    R Tlo;
    const R T = heat_of(g, Tlo);
    R p, dpdT, inv_rho;
    eos(rho, T, P, p, dpdT, &inv_rho);
    const R psi2 = psi_squared(p, dpdT, Tlo, rho, C);
    const int bad = classify(rho, T, psi2, P);
    if (bad) report(status, step, x, y, bad);
    pl.p[P_RHO][i] = rho;
    pl.p[P_T][i] = T;
    pl.p[P_PSI][i] = sqrt(fmax(psi2, R(0)));
    pl.p[P_JX][i] = jx;
    pl.p[P_JY][i] = jy;
    pl.p[P_DPDT][i] = dpdT;
    pl.p[P_IRHO][i] = inv_rho;
    if (do_partials) rho_d = (double)rho;
  }
  if (do_partials) {
    const double s = block_sum<BLOCK>(rho_d, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
  }
}

template <class R>
__global__ void __launch_bounds__(BLOCK) k_force(Planes<R> pl, DevParams P, const double* __restrict__ rho_ave) {
  const Coefs<R>& C = coefs<R>(P);
  const long long i = (long long)blockIdx.x * BLOCK + threadIdx.x;
  if (i >= P.N) return;
  const int y = (int)(i / P.nx), x = (int)(i - (long long)y * P.nx);
  const R* __restrict__ psi = pl.p[P_PSI];
  R c[3][3];
  gather9(psi, P, x, y, c);
  // F_int = -G psi(x) sum_a w(|e_a|^2) psi(x+e_a) e_a, w(1) = 1/3, w(2) = 1/12; ghost rows beyond a
  // non-periodic edge copy the edge row, so a wall with G_wall = 0 is neutral.
  const R pc = psi[i];
  const R sx = (c[1][2] - c[1][0]) * R(1.0 / 3.0) + (c[2][2] - c[2][0] - c[0][0] + c[0][2]) * R(1.0 / 12.0);
  const R sy = (c[2][1] - c[0][1]) * R(1.0 / 3.0) + (c[2][2] + c[2][0] - c[0][0] - c[0][2]) * R(1.0 / 12.0);
  const R Fix = -C.G * pc * sx, Fiy = -C.G * pc * sy;
  R Fx = Fix, Fy = Fiy;
  // F_ads = -G_w psi(x) sum_a w_a psi(x) s(x+e_a) e_a on the y- wall, whose solid ghost row gives the
  // sum (0, -1/2). A y+ wall is a neutral lid (the solid surfaces of Sec. IV are bottom walls).
  if (!P.yper && y == 0 && P.ybc_lo == BC_WALL) Fy += C.G_wall * 0.5f * pc * pc;
  const R rho = pl.p[P_RHO][i];
  if (P.buoyancy) {  // F_b = (rho - rho_ref) g: rho_ref = rho_ave (Sec. IV B) or the y+ edge's held density
    const R dr = rho - (P.buoyancy == 1 ? R(*rho_ave) : C.rho_bc_hi);
    Fx += dr * C.gx;
    Fy += dr * C.gy;
  }
  const R inv_rho = pl.p[P_IRHO][i];
  pl.p[P_VX][i] = (pl.p[P_JX][i] + Fx * 0.5f) * inv_rho;
  pl.p[P_VY][i] = (pl.p[P_JY][i] + Fy * 0.5f) * inv_rho;
  pl.p[P_FX][i] = Fx;
  pl.p[P_FY][i] = Fy;
  // sigma term Q = qcoef |F_int|^2 / psi^2 = qcoef G^2 (sx^2 + sy^2): psi^2 cancels
  pl.p[P_Q][i] = C.qG2 * (sx * sx + sy * sy);
}

// Two warp-uniform roles per node: the first BLOCK threads of a block run the flow collision of
// BLOCK nodes, the next BLOCK threads run the source and thermal collision of the same nodes. The
// roles share no data (both read the scratch planes), so a node's work splits into two independent
// chains and twice as many warps hide the FP64 latency on small grids.
//
// BY_BLOCK = false: each block of 2 * BLOCK threads holds both roles of BLOCK nodes. BY_BLOCK = true:
// blocks of BLOCK threads, the first half of the grid runs the flow role and the second half the
// thermal role. Blocks start roughly in index order, so an SM then runs one role's code at a time,
// which keeps long double-word code (LBPC_DF64) in the instruction caches.
template <class S, class R, bool BY_BLOCK>
__global__ void __launch_bounds__(BY_BLOCK ? BLOCK : 2 * BLOCK)
    k_collide(PopBuf<S> fsrc, PopBuf<S> gsrc, PopBuf<S> fdst, PopBuf<S> gdst, Planes<R> pl, R* __restrict__ phi_prev,
              DevParams P, int first) {
  const Coefs<R>& C = coefs<R>(P);
  const unsigned half = gridDim.x >> 1;
  const bool heat = BY_BLOCK ? blockIdx.x >= half : threadIdx.x >= BLOCK;
  const long long i = BY_BLOCK ? (long long)(blockIdx.x - (heat ? half : 0u)) * BLOCK + threadIdx.x
                               : (long long)blockIdx.x * BLOCK + (threadIdx.x - (heat ? BLOCK : 0));
  if (i >= P.N) return;
  const int y = (int)(i / P.nx), x = (int)(i - (long long)y * P.nx);
  const R vx = pl.p[P_VX][i], vy = pl.p[P_VY][i];
  if (!heat) {
    R f[9];
    pull<S, R>(fsrc, C.wf, P, x, y, f);
    flow_closure(f, P, x, y, fsrc.wall);
    const R rho = pl.p[P_RHO][i];
    const R Fx = pl.p[P_FX][i], Fy = pl.p[P_FY][i];
    collide_flow(f, rho, vx, vy, Fx, Fy, pl.p[P_Q][i], P);
    pop_store<S, R>(fdst, P.N, i, f, rho, C.wf);
    wall_force_store(fdst.wall, P, x, y, Fx, Fy);
    return;
  }
  R g[9];
  pull<S, R>(gsrc, C.wg, P, x, y, g);
  heat_closure(g, P, x, y);
  const R rho = pl.p[P_RHO][i];
  const R T = pl.p[P_T][i];
  // gradients feeding the source (isotropic differences)
  R c[3][3];
  gather9(pl.p[P_T], P, x, y, c);
  const R gTx = d_x(c), gTy = d_y(c), lapT = lap(c);
  gather9(pl.p[P_VX], P, x, y, c);
  R divv = d_x(c);
  gather9(pl.p[P_VY], P, x, y, c);
  divv += d_y(c);
  const R rcv = rho * C.cV;
  const R inv_rcv = pl.p[P_IRHO][i] * C.inv_cV;
  R div_lam_gradT;
  if (P.lambda_mode == 0) {
    div_lam_gradT = C.lambda * lapT;
  } else {  // lambda = rho c_V chi: lambda lap T + c_V chi grad rho . grad T
    gather9(pl.p[P_RHO], P, x, y, c);
    div_lam_gradT = rcv * C.chi * lapT + C.cV_chi * (d_x(c) * gTx + d_y(c) * gTy);
  }
  const R compress = T * (R(1) - pl.p[P_DPDT][i] * inv_rcv) * divv;
  R phi, S0, tau_inv = R(0);
  if (P.model == 2) {
    // Gong-Cheng: the source is Eq. 13 alone; tau_g = lambda/(rho c_s^2 c_V) + 1/2 (Sec. IV A)
    phi = compress;
    S0 = phi;
    tau_inv = R(1) / ((P.lambda_mode == 0 ? C.lambda * 3 * inv_rcv : C.chi * 3) + R(0.5));
  } else {
    // phi: the underlined terms of Eq. 28 with k = (1/s_3 - 1/2) c_s^2
    phi = div_lam_gradT * inv_rcv - C.kdiff * lapT + compress;
    S0 = phi;
    if (P.model == 0) {  // S0 = phi + 0.5 dt d_t phi, d_t phi ~ [phi(t) - phi(t - dt)]/dt (Eq. 46)
      const R pp = first ? phi : phi_prev[i];
      S0 = phi + (phi - pp) * 0.5f;
    }
  }
  phi_prev[i] = phi;
  collide_heat(g, T, vx, vy, S0, P, tau_inv);
  pop_store<S, R>(gdst, P.N, i, g, T + S0, C.wg);
}

// Fixed-order sum of the block partials: each thread accumulates a strided subset in order, then one
// block reduction. out[k] = sum(partials[k * stride + 0 .. n)) * scale.
__global__ void __launch_bounds__(BLOCK) k_finish(const double* __restrict__ partials, int n, int stride, int count,
                                                  double scale, double* __restrict__ out) {
  __shared__ double red[BLOCK / 32];
  for (int k = 0; k < count; ++k) {
    double s = 0.0;
    for (int j = threadIdx.x; j < n; j += BLOCK) s += partials[(long long)k * stride + j];
    s = block_sum<BLOCK>(s, red);
    if (threadIdx.x == 0) out[k] = s * scale;
  }
}

// Equilibrium start: writes post-collision-layout buffers whose pull gives f = M^{-1} m_eq(rho, u),
// g = M^{-1} m_eq(T, u) at every node (the slot that node x pulls for direction a sits at x - e_a).
template <class S>
__global__ void __launch_bounds__(BLOCK) k_init(const double* __restrict__ rho_in, const double* __restrict__ T_in,
                                                const double* __restrict__ ux_in, const double* __restrict__ uy_in,
                                                PopBuf<S> f, PopBuf<S> g, DevParams P) {
  const long long i = (long long)blockIdx.x * BLOCK + threadIdx.x;
  if (i >= P.N) return;
  const int y = (int)(i / P.nx), x = (int)(i - (long long)y * P.nx);
  double fv[9], gv[9];
#pragma unroll
  for (int a = 0; a < 9; ++a) {
    // node whose pull reads slot (x, y) in direction a
    const int tx = wrapx(x + EX(a), P.nx);
    int ty = y + EY(a);
    if (ty < 0 || ty >= P.ny) {
      if (!P.yper) {  // no node pulls this slot; keep it finite
        fv[a] = 0.0;
        gv[a] = 0.0;
        continue;
      }
      ty = ty < 0 ? ty + P.ny : ty - P.ny;
    }
    const long long t = (long long)ty * P.nx + tx;
    const double rho = rho_in[t], T = T_in[t];
    const double vx = ux_in ? ux_in[t] : 0.0, vy = uy_in ? uy_in[t] : 0.0;
    const double v2 = vx * vx + vy * vy;
    double m[9], fe[9], ge[9];
    m[0] = rho; m[1] = rho * (-2.0 + 3.0 * v2); m[2] = rho * (1.0 - 3.0 * v2);
    m[3] = rho * vx; m[4] = -rho * vx; m[5] = rho * vy; m[6] = -rho * vy;
    m[7] = rho * (vx * vx - vy * vy); m[8] = rho * vx * vy;
    from_moments(m, fe);
    heat_meq(T, vx, vy, P.model, m);
    from_moments(m, ge);
    fv[a] = fe[a];
    gv[a] = ge[a];
  }
  // FP16 storage: deviations from the rest equilibrium of this slot's own node
  pop_store<S, double>(f, P.N, i, fv, rho_in[i], P.cd.wf);
  pop_store<S, double>(g, P.N, i, gv, T_in[i], P.cd.wg);
}

// Sums of rho and T over the current (post-boundary) state into per-block partials.
template <class S>
__global__ void __launch_bounds__(BLOCK) k_sums(PopBuf<S> fsrc, PopBuf<S> gsrc, DevParams P,
                                                double* __restrict__ partials, int stride) {
  __shared__ double red[BLOCK / 32];
  const long long i = (long long)blockIdx.x * BLOCK + threadIdx.x;
  double r = 0.0, t = 0.0;
  if (i < P.N) {
    const int y = (int)(i / P.nx), x = (int)(i - (long long)y * P.nx);
    double f[9], g[9];
    pull_closed<S, double>(fsrc, gsrc, P, x, y, f, g);
    r = f[0] + f[1] + f[2] + f[3] + f[4] + f[5] + f[6] + f[7] + f[8];
    t = g[0] + g[1] + g[2] + g[3] + g[4] + g[5] + g[6] + g[7] + g[8];
  }
  const double sr = block_sum<BLOCK>(r, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = sr;
  const double st = block_sum<BLOCK>(t, red);
  if (threadIdx.x == 0) partials[stride + blockIdx.x] = st;
}

// Post-boundary populations of the current state as FP64 [9][N] (which = 0: f, 1: g).
template <class S>
__global__ void __launch_bounds__(BLOCK) k_export_pops(PopBuf<S> fsrc, PopBuf<S> gsrc, DevParams P, int which,
                                                       int only, double* __restrict__ out) {
  const long long i = (long long)blockIdx.x * BLOCK + threadIdx.x;
  if (i >= P.N) return;
  const int y = (int)(i / P.nx), x = (int)(i - (long long)y * P.nx);
  double f[9], g[9];
  pull_closed<S, double>(fsrc, gsrc, P, x, y, f, g);
  if (only >= 0) {  // one population plane into out[N]
    out[i] = which ? g[only] : f[only];
    return;
  }
#pragma unroll
  for (int a = 0; a < 9; ++a) out[(long long)a * P.N + i] = which ? g[a] : f[a];
}

// Copy planes rho, vx, vy, T to FP64 outputs (any may be null).
template <class R>
__global__ void __launch_bounds__(BLOCK) k_export_fields(Planes<R> pl, DevParams P, double* rho, double* ux, double* uy,
                                                         double* T) {
  const long long i = (long long)blockIdx.x * BLOCK + threadIdx.x;
  if (i >= P.N) return;
  if (rho) rho[i] = (double)pl.p[P_RHO][i];
  if (ux) ux[i] = (double)pl.p[P_VX][i];
  if (uy) uy[i] = (double)pl.p[P_VY][i];
  if (T) T[i] = (double)pl.p[P_T][i];
}

// ------------------------------------------------------------------------------------------------
// host launchers
// ------------------------------------------------------------------------------------------------
static inline unsigned blocks_for(long long N) { return (unsigned)((N + BLOCK - 1) / BLOCK); }

template <class S, class R> static Planes<R> planes_of(const SplitBuffers& b) {
  Planes<R> pl;
  for (int k = 0; k < NPLANES; ++k) pl.p[k] = (R*)b.planes[k];
  return pl;
}

template <class S> static PopBuf<S> fbuf(const SplitBuffers& b, int k) {
  return PopBuf<S>{(S*)b.f[k], b.ref_f[k], b.wall[k]};
}
template <class S> static PopBuf<S> gbuf(const SplitBuffers& b, int k) { return PopBuf<S>{(S*)b.g[k], b.ref_g[k]}; }

// Role layout of k_collide per storage type (both compute the same step): roles by block for the
// long double-word code (measured 15 % faster at 2048^2), roles within a block otherwise.
template <class S> static constexpr bool collide_by_block() { return is_dw_t<S>::value; }

template <class S, class R>
static cudaError_t step_impl(const SplitBuffers& b, const DevParams& P, int cur, long long step, cudaStream_t st,
                             cudaEvent_t* ev) {
  const unsigned nb = blocks_for(P.N);
  Planes<R> pl = planes_of<S, R>(b);
  if (ev) cudaEventRecord(ev[0], st);
  k_macro<S, R><<<nb, BLOCK, 0, st>>>(fbuf<S>(b, cur), gbuf<S>(b, cur), pl, P, step, P.buoyancy == 1, b.partials, b.status);
  if (ev) cudaEventRecord(ev[1], st);
  k_force<R><<<nb, BLOCK, 0, st>>>(pl, P, b.scalars);
  if (ev) cudaEventRecord(ev[2], st);
  if (collide_by_block<S>())
    k_collide<S, R, true><<<2 * nb, BLOCK, 0, st>>>(fbuf<S>(b, cur), gbuf<S>(b, cur), fbuf<S>(b, cur ^ 1),
                                                   gbuf<S>(b, cur ^ 1), pl, (R*)b.phi_prev, P, step == 0);
  else
    k_collide<S, R, false><<<nb, 2 * BLOCK, 0, st>>>(fbuf<S>(b, cur), gbuf<S>(b, cur), fbuf<S>(b, cur ^ 1),
                                                    gbuf<S>(b, cur ^ 1), pl, (R*)b.phi_prev, P, step == 0);
  if (ev) cudaEventRecord(ev[3], st);
  if (P.buoyancy == 1) {
    k_finish<<<1, BLOCK, 0, st>>>(b.partials, (int)nb, 0, 1, 1.0 / (double)P.N, b.scalars);
    if (ev) cudaEventRecord(ev[4], st);
  }
  return cudaGetLastError();
}

cudaError_t split_step(const SplitBuffers& b, const DevParams& P, int prec, int cur, long long step, cudaStream_t st,
                       cudaEvent_t* ev) {
  if (prec == 0) return step_impl<double, double>(b, P, cur, step, st, ev);
  if (prec == 1) return step_impl<float, float>(b, P, cur, step, st, ev);
  if (prec == 3) return step_impl<dw, dw>(b, P, cur, step, st, ev);
  return step_impl<__half, float>(b, P, cur, step, st, ev);
}

int split_kernel_count(const DevParams& P) { return P.buoyancy == 1 ? 4 : 3; }

const char* split_kernel_name(int k) {
  static const char* names[] = {"k_macro", "k_force", "k_collide", "k_finish"};
  return (k >= 0 && k < 4) ? names[k] : "";
}

template <class S>
static cudaError_t init_impl(const SplitBuffers& b, const DevParams& P, const double* rho, const double* T,
                             const double* ux, const double* uy, cudaStream_t st) {
  const unsigned nb = blocks_for(P.N);
  for (int k = 0; k < 2; ++k)  // no force before the first step: the initial closure takes j = 0 on walls
    if (b.wall[k]) {
      const cudaError_t e = cudaMemsetAsync(b.wall[k], 0, wall_doubles(P.nx) * sizeof(double), st);
      if (e != cudaSuccess) return e;
    }
  k_init<S><<<nb, BLOCK, 0, st>>>(rho, T, ux, uy, fbuf<S>(b, 0), gbuf<S>(b, 0), P);
  // rho_ave of the initial (post-boundary) state
  k_sums<S><<<nb, BLOCK, 0, st>>>(fbuf<S>(b, 0), gbuf<S>(b, 0), P, b.partials, (int)nb);
  k_finish<<<1, BLOCK, 0, st>>>(b.partials, (int)nb, (int)nb, 1, 1.0 / (double)P.N, b.scalars);
  return cudaGetLastError();
}

cudaError_t split_init(const SplitBuffers& b, const DevParams& P, int prec, const double* rho, const double* T,
                       const double* ux, const double* uy, cudaStream_t st) {
  if (prec == 0) return init_impl<double>(b, P, rho, T, ux, uy, st);
  if (prec == 1) return init_impl<float>(b, P, rho, T, ux, uy, st);
  if (prec == 3) return init_impl<dw>(b, P, rho, T, ux, uy, st);
  return init_impl<__half>(b, P, rho, T, ux, uy, st);
}

template <class S>
static cudaError_t sums_impl(const SplitBuffers& b, const DevParams& P, int cur, cudaStream_t st) {
  const unsigned nb = blocks_for(P.N);
  k_sums<S><<<nb, BLOCK, 0, st>>>(fbuf<S>(b, cur), gbuf<S>(b, cur), P, b.partials, (int)nb);
  k_finish<<<1, BLOCK, 0, st>>>(b.partials, (int)nb, (int)nb, 2, 1.0, b.scalars + 1);
  return cudaGetLastError();
}

cudaError_t split_sums(const SplitBuffers& b, const DevParams& P, int prec, int cur, cudaStream_t st) {
  if (prec == 0) return sums_impl<double>(b, P, cur, st);
  if (prec == 1) return sums_impl<float>(b, P, cur, st);
  if (prec == 3) return sums_impl<dw>(b, P, cur, st);
  return sums_impl<__half>(b, P, cur, st);
}

template <class S, class R>
static cudaError_t fields_impl(const SplitBuffers& b, const DevParams& P, int cur, long long step, double* rho,
                               double* ux, double* uy, double* T, cudaStream_t st) {
  const unsigned nb = blocks_for(P.N);
  Planes<R> pl = planes_of<S, R>(b);
  k_macro<S, R><<<nb, BLOCK, 0, st>>>(fbuf<S>(b, cur), gbuf<S>(b, cur), pl, P, step, 0, b.partials, b.status);
  k_force<R><<<nb, BLOCK, 0, st>>>(pl, P, b.scalars);
  k_export_fields<R><<<nb, BLOCK, 0, st>>>(pl, P, rho, ux, uy, T);
  return cudaGetLastError();
}

cudaError_t split_fields(const SplitBuffers& b, const DevParams& P, int prec, int cur, long long step, double* rho,
                         double* ux, double* uy, double* T, cudaStream_t st) {
  if (prec == 0) return fields_impl<double, double>(b, P, cur, step, rho, ux, uy, T, st);
  if (prec == 1) return fields_impl<float, float>(b, P, cur, step, rho, ux, uy, T, st);
  if (prec == 3) return fields_impl<dw, dw>(b, P, cur, step, rho, ux, uy, T, st);
  return fields_impl<__half, float>(b, P, cur, step, rho, ux, uy, T, st);
}

cudaError_t split_export_pops(const SplitBuffers& b, const DevParams& P, int prec, int cur, int which, int only,
                              double* out, cudaStream_t st) {
  const unsigned nb = blocks_for(P.N);
  if (prec == 0)
    k_export_pops<double><<<nb, BLOCK, 0, st>>>(fbuf<double>(b, cur), gbuf<double>(b, cur), P, which, only, out);
  else if (prec == 1)
    k_export_pops<float><<<nb, BLOCK, 0, st>>>(fbuf<float>(b, cur), gbuf<float>(b, cur), P, which, only, out);
  else if (prec == 3)
    k_export_pops<dw><<<nb, BLOCK, 0, st>>>(fbuf<dw>(b, cur), gbuf<dw>(b, cur), P, which, only, out);
  else
    k_export_pops<__half><<<nb, BLOCK, 0, st>>>(fbuf<__half>(b, cur), gbuf<__half>(b, cur), P, which, only, out);
  return cudaGetLastError();
}

void fused_finish(const SplitBuffers& b, const DevParams& P, int n, cudaStream_t st) {
  k_finish<<<1, BLOCK, 0, st>>>(b.partials, n, 0, 1, 1.0 / (double)P.N, b.scalars);
}

int split_nplanes() { return NPLANES; }
int split_block() { return BLOCK; }

}  // namespace lbpc
