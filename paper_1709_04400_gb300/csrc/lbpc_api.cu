// C ABI of liblbpc (declared in include/lbpc.h): parameter validation, workspace layout, the context
// and the host-side EOS helpers. The compute runs in the kernels of lbpc_split.cu.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "../../include/lbpc.h"
#include "lbpc_internal.h"

#define LBPC_API extern "C" __attribute__((visibility("default")))

using lbpc::DevParams;
using lbpc::SplitBuffers;

struct lbpc_ctx {
  lbpc_params p;
  DevParams dp;
  int device;
  cudaStream_t stream;
  SplitBuffers buf;
  int cur;              // buffer holding the current state
  int path;             // lbpc_path
  size_t stage_bytes;   // bytes of one A/B half (f and g): the FP64 staging room between steps
  long long step;
  int initialised;
  lbpc::TmaMaps tma[2];  // tensor maps of buffers A and B (TMA-staged fused step)
  cudaEvent_t ev[8];    // created on first lbpc_step_timed
  int have_events;
  lbpc_status err;
  char msg[512];
};

namespace {

struct DeviceGuard {
  int old = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&old) == cudaSuccess && old != dev) cudaSetDevice(dev);
    else old = -1;
  }
  ~DeviceGuard() {
    if (old >= 0) cudaSetDevice(old);
  }
};

void set_msg(char* dst, size_t n, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
void set_msg(char* dst, size_t n, const char* fmt, ...) {
  if (!dst || n == 0) return;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, n, fmt, ap);
  va_end(ap);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
  size_t f[2], g[2], ref_f[2], ref_g[2], wall[2], phi, planes, partials, scalars, status, total;
  size_t store, real;
  long long N;
  int nblocks;
};

Layout layout_of(const lbpc_params* p) {
  Layout L{};
  L.N = (long long)p->nx * p->ny;
  L.store = (p->prec == LBPC_FP64 || p->prec == LBPC_DF64) ? 8 : (p->prec == LBPC_FP32 ? 4 : 2);
  L.real = (p->prec == LBPC_FP64 || p->prec == LBPC_DF64) ? 8 : 4;
  L.nblocks = (int)((L.N + lbpc::split_block() - 1) / lbpc::split_block());
  size_t off = 0;
  const size_t pop = align256(9 * (size_t)L.N * L.store);
  // f0 g0 f1 g1: each A/B half is contiguous so the dead half can stage FP64 transfers
  L.f[0] = off; off += pop;
  L.g[0] = off; off += pop;
  L.f[1] = off; off += pop;
  L.g[1] = off; off += pop;
  const size_t ref = p->prec == LBPC_FP16DEV ? align256((size_t)L.N * sizeof(float)) : 0;
  for (int k = 0; k < 2; ++k) {
    L.ref_f[k] = off; off += ref;
    L.ref_g[k] = off; off += ref;
  }
  for (int k = 0; k < 2; ++k) {  // wall-row forces kept with f (A/B) for the next step's wall closure
    L.wall[k] = off; off += align256((size_t)lbpc::wall_doubles(p->nx) * sizeof(double));
  }
  L.phi = off; off += align256((size_t)L.N * L.real);
  L.planes = off; off += (size_t)lbpc::split_nplanes() * align256((size_t)L.N * L.real);
  // per-block partials of the split step, or per-tile partials of the fused step (more on narrow domains)
  const size_t npartials = 2 * (size_t)L.nblocks > lbpc::fused_max_tiles(p->nx, p->ny)
                               ? 2 * (size_t)L.nblocks : lbpc::fused_max_tiles(p->nx, p->ny);
  L.partials = off; off += align256(npartials * sizeof(double));
  L.scalars = off; off += align256(8 * sizeof(double));
  L.status = off; off += align256(8 * sizeof(long long));
  L.total = off;
  return L;
}

lbpc_status fail(lbpc_ctx* c, lbpc_status s, const char* what) {
  if (c->err == LBPC_OK) {
    c->err = s;
    set_msg(c->msg, sizeof c->msg, "%s", what);
  }
  return s;
}

lbpc_status cuda_fail(lbpc_ctx* c, cudaError_t e, const char* where) {
  char m[400];
  snprintf(m, sizeof m, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
  return fail(c, LBPC_ECUDA, m);
}

#define CU(c, call, where)                              \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
  } while (0)

bool is_dirichlet_ok(int v) { return v == LBPC_T_NONE || v == LBPC_T_DIRICHLET; }

double critical_T(const lbpc_params* p) { return 0.0778 * p->a / (0.45724 * p->b * p->R); }
double kappa_of(double om) { return 0.37464 + 1.54226 * om - 0.26992 * om * om; }

template <class R> void fill_coefs(lbpc::Coefs<R>& c, const lbpc_params* p) {
  for (int k = 0; k < 4; ++k) c.T_bc[k] = (R)p->T_bc[k];
  c.T_strip = (R)p->T_strip;
  c.rho_bc_lo = (R)p->rho_bc[2];
  c.rho_bc_hi = (R)p->rho_bc[3];
  c.a = (R)p->a;
  c.b = (R)p->b;
  c.R_gas = (R)p->R;
  c.G = (R)p->G;
  c.kappa = (R)kappa_of(p->omega);
  for (int k = 0; k < 9; ++k) {
    c.s_f[k] = (R)p->s_f[k];
    c.s_g[k] = (R)p->s_g[k];
    c.hf[k] = (R)(1.0 - 0.5 * p->s_f[k]);
  }
  c.lambda = (R)p->lambda;
  c.chi = (R)p->chi;
  c.cV = (R)p->cV;
  c.kdiff = (R)((1.0 / p->s_g[3] - 0.5) / 3.0);
  c.gx = (R)p->gx;
  c.gy = (R)p->gy;
  c.G_wall = (R)p->G_wall;
  c.c3 = (R)((1.0 - 0.5 * p->s_g[3]) * p->s_g[4]);
  c.c5 = (R)((1.0 - 0.5 * p->s_g[5]) * p->s_g[6]);
  c.inv_Tc = (R)(1.0 / critical_T(p));
  c.qG2 = (R)(12.0 * p->sigma / (1.0 / p->s_f[1] - 0.5) * p->G * p->G);
  c.inv_cV = (R)(1.0 / p->cV);
  c.psi_scale = (R)(2.0 / p->G);
  c.cV_chi = (R)(p->cV * p->chi);
  // rest-state equilibrium weights: f at rest is w_a rho; g at rest is M^{-1} m_eq(T, 0), which for
  // Eq. 53 (m2_eq = 2T) is (5/9, 1/18 x8) and for Eq. 44 (m2_eq = T) the D2Q9 weights
  const double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
  const double wi[9] = {5.0 / 9, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18};
  for (int k = 0; k < 9; ++k) {
    c.wf[k] = (R)w[k];
    c.wg[k] = (R)(p->model == LBPC_IMPROVED ? wi[k] : w[k]);
  }
}

DevParams make_dev_params(const lbpc_params* p) {
  DevParams d{};
  d.nx = p->nx;
  d.ny = p->ny;
  d.N = (long long)p->nx * p->ny;
  d.yper = p->flow_bc[2] == LBPC_PERIODIC;
  d.ybc_lo = p->flow_bc[2];
  d.ybc_hi = p->flow_bc[3];
  for (int k = 0; k < 4; ++k) d.tbc[k] = p->t_bc[k];
  d.strip_x0 = p->strip_x0;
  d.strip_x1 = p->strip_x1;
  d.model = p->model;
  d.lambda_mode = p->lambda_mode;
  d.buoyancy = p->buoyancy;  // 0 none, 1 reference rho_ave, 2 reference rho_bc of the y+ edge
  d.heat_unit_rates = 1;
  for (int k = 1; k < 9; ++k) d.heat_unit_rates &= p->s_g[k] == 1.0;
  fill_coefs(d.cd, p);
  fill_coefs(d.cf, p);
  fill_coefs(d.cw, p);
  return d;
}

// ---- Peng-Robinson helpers on the host (Eq. 56) ----
double pr_pressure(const lbpc_params* p, double rho, double T) {
  const double Tc = critical_T(p), k = kappa_of(p->omega);
  const double th = 1.0 + k * (1.0 - sqrt(T / Tc));
  return rho * p->R * T / (1.0 - p->b * rho) - p->a * th * th * rho * rho / (1.0 + 2.0 * p->b * rho - p->b * p->b * rho * rho);
}

double pr_dp_drho(const lbpc_params* p, double rho, double T) {
  const double Tc = critical_T(p), k = kappa_of(p->omega);
  const double th = 1.0 + k * (1.0 - sqrt(T / Tc));
  const double d = 1.0 + 2.0 * p->b * rho - p->b * p->b * rho * rho;
  return p->R * T / ((1.0 - p->b * rho) * (1.0 - p->b * rho)) - p->a * th * th * 2.0 * rho * (1.0 + p->b * rho) / (d * d);
}

// ln of the Peng-Robinson fugacity coefficient at compressibility Z (pure fluid).
double pr_ln_phi(const lbpc_params* p, double T, double P, double rho) {
  const double Tc = critical_T(p), k = kappa_of(p->omega);
  const double th = 1.0 + k * (1.0 - sqrt(T / Tc));
  const double A = p->a * th * th * P / (p->R * T * p->R * T), B = p->b * P / (p->R * T);
  const double Z = P / (rho * p->R * T);
  const double s2 = sqrt(2.0);
  return (Z - 1.0) - log(Z - B) - A / (2.0 * s2 * B) * log((Z + (1.0 + s2) * B) / (Z + (1.0 - s2) * B));
}

template <class F> double bisect(F fn, double lo, double hi) {
  double flo = fn(lo);
  for (int it = 0; it < 400 && hi - lo > 1e-16 * fmax(1.0, fabs(lo)); ++it) {
    const double mid = 0.5 * (lo + hi), fm = fn(mid);
    if ((fm > 0) == (flo > 0)) { lo = mid; flo = fm; } else { hi = mid; }
  }
  return 0.5 * (lo + hi);
}

}  // namespace

namespace lbpc {
DevParams make_dev_params_public(const lbpc_params* p) { return make_dev_params(p); }
}  // namespace lbpc

// ================================================================================================
// exported
// ================================================================================================

LBPC_API int32_t lbpc_version(void) { return LBPC_VERSION; }

LBPC_API lbpc_status lbpc_check_params(const lbpc_params* p, char* msg, size_t n) {
#define BAD(...)                    \
  do {                              \
    set_msg(msg, n, __VA_ARGS__);   \
    return LBPC_EINVAL;             \
  } while (0)
  if (!p) BAD("params is NULL");
  if (p->nx < 2 || p->ny < 2) BAD("grid %d x %d: nx and ny must be >= 2", p->nx, p->ny);
  if ((long long)p->nx * p->ny > (1ll << 31)) BAD("grid %d x %d exceeds 2^31 nodes", p->nx, p->ny);
  if (p->prec != LBPC_FP64 && p->prec != LBPC_FP32 && p->prec != LBPC_FP16DEV && p->prec != LBPC_DF64)
    BAD("prec %d unknown", p->prec);
  if (p->model != LBPC_IMPROVED && p->model != LBPC_COMPROMISED && p->model != LBPC_GONG_CHENG)
    BAD("model %d unknown", p->model);
  if (p->lambda_mode != LBPC_LAMBDA_CONST && p->lambda_mode != LBPC_LAMBDA_RHO_CV_CHI) BAD("lambda_mode %d unknown", p->lambda_mode);
  if (p->flow_bc[0] != LBPC_PERIODIC || p->flow_bc[1] != LBPC_PERIODIC) BAD("x edges must be periodic");
  for (int k = 2; k < 4; ++k)
    if (p->flow_bc[k] != LBPC_PERIODIC && p->flow_bc[k] != LBPC_WALL && p->flow_bc[k] != LBPC_PRESSURE)
      BAD("flow_bc[%d] = %d unknown", k, p->flow_bc[k]);
  if ((p->flow_bc[2] == LBPC_PERIODIC) != (p->flow_bc[3] == LBPC_PERIODIC))
    BAD("y edges must be both periodic or both non-periodic");
  if (p->flow_bc[2] != LBPC_PERIODIC && p->ny < 3) BAD("non-periodic y needs ny >= 3");
  for (int k = 0; k < 4; ++k) {
    if (!is_dirichlet_ok(p->t_bc[k])) BAD("t_bc[%d] = %d unknown", k, p->t_bc[k]);
    if (p->t_bc[k] == LBPC_T_DIRICHLET && !(p->T_bc[k] > 0)) BAD("T_bc[%d] must be > 0", k);
    if (k >= 2 && p->flow_bc[k] == LBPC_PRESSURE && !(p->rho_bc[k] > 0)) BAD("rho_bc[%d] must be > 0", k);
  }
  if (p->strip_x1 != p->strip_x0) {
    if (p->strip_x0 < 0 || p->strip_x1 < p->strip_x0 || p->strip_x1 > p->nx) BAD("strip [%d, %d) outside 0..nx", p->strip_x0, p->strip_x1);
    if (p->t_bc[2] != LBPC_T_DIRICHLET) BAD("a heated strip needs t_bc[2] = LBPC_T_DIRICHLET");
    if (!(p->T_strip > 0)) BAD("T_strip must be > 0");
  }
  if (!(p->a > 0) || !(p->b > 0) || !(p->R > 0)) BAD("a, b, R must be > 0");
  if (!(p->G != 0) || !isfinite(p->G)) BAD("G must be finite and nonzero");
  for (int k = 0; k < 9; ++k) {
    if (!(p->s_f[k] > 0 && p->s_f[k] < 2)) BAD("s_f[%d] = %g outside (0, 2)", k, p->s_f[k]);
    if (!(p->s_g[k] > 0 && p->s_g[k] < 2)) BAD("s_g[%d] = %g outside (0, 2)", k, p->s_g[k]);
  }
  if (!(p->cV > 0)) BAD("cV must be > 0");
  if (p->lambda_mode == LBPC_LAMBDA_CONST && !(p->lambda > 0)) BAD("lambda must be > 0");
  if (p->lambda_mode == LBPC_LAMBDA_RHO_CV_CHI && !(p->chi > 0)) BAD("chi must be > 0");
  if (!isfinite(p->sigma) || !isfinite(p->gx) || !isfinite(p->gy) || !isfinite(p->G_wall)) BAD("non-finite parameter");
  if (p->buoyancy < 0 || p->buoyancy > 2) BAD("buoyancy %d unknown", p->buoyancy);
  if (p->buoyancy == 2 && p->flow_bc[3] != LBPC_PRESSURE) BAD("buoyancy 2 needs a fixed-density y+ edge");
  set_msg(msg, n, "ok");
  return LBPC_OK;
#undef BAD
}

LBPC_API size_t lbpc_workspace_bytes(const lbpc_params* p) {
  if (lbpc_check_params(p, nullptr, 0) != LBPC_OK) return 0;
  return layout_of(p).total;
}

LBPC_API lbpc_status lbpc_eos_critical(const lbpc_params* p, double* Tc, double* pc) {
  if (!p || !(p->a > 0) || !(p->b > 0) || !(p->R > 0)) return LBPC_EINVAL;
  const double t = critical_T(p);
  if (Tc) *Tc = t;
  if (pc) *pc = 0.0778 * p->R * t / p->b;
  return LBPC_OK;
}

LBPC_API lbpc_status lbpc_coexistence(const lbpc_params* p, double T, double* rho_v, double* rho_l, double* p_sat) {
  if (!p || !(p->a > 0) || !(p->b > 0) || !(p->R > 0)) return LBPC_EINVAL;
  const double Tc = critical_T(p);
  if (!(T > 0) || !(T < Tc)) return LBPC_EINVAL;
  // spinodals: sign changes of (dp/drho)_T on a fine grid, refined by bisection
  const double rmax = 1.0 / p->b;
  const int n = 20000;
  double sp[2];
  int ns = 0;
  double prev = pr_dp_drho(p, rmax * 1e-6, T);
  for (int i = 1; i < n && ns < 2; ++i) {
    const double r0 = rmax * (1e-6 + (1 - 2e-6) * (i - 1) / (n - 1)), r1 = rmax * (1e-6 + (1 - 2e-6) * i / (n - 1));
    const double cur = pr_dp_drho(p, r1, T);
    if ((cur > 0) != (prev > 0)) sp[ns++] = bisect([&](double r) { return pr_dp_drho(p, r, T); }, r0, r1);
    prev = cur;
  }
  if (ns != 2) return LBPC_EINVAL;
  auto roots = [&](double ps, double& rv, double& rl) {
    rv = bisect([&](double r) { return pr_pressure(p, r, T) - ps; }, fmin(1e-12, 0.5 * ps / (p->R * T)), sp[0]);
    rl = bisect([&](double r) { return pr_pressure(p, r, T) - ps; }, sp[1], rmax * (1.0 - 1e-12));
  };
  const double phi_hi = pr_pressure(p, sp[0], T);
  const double plo = fmax(pr_pressure(p, sp[1], T), 1e-300);
  // coexistence: equal fugacity of the two outer roots at the same pressure
  const double ps = bisect(
      [&](double P) {
        double rv, rl;
        roots(P, rv, rl);
        return pr_ln_phi(p, T, P, rv) - pr_ln_phi(p, T, P, rl);
      },
      plo + 1e-14 * phi_hi, phi_hi * (1 - 1e-14));
  double rv, rl;
  roots(ps, rv, rl);
  if (rho_v) *rho_v = rv;
  if (rho_l) *rho_l = rl;
  if (p_sat) *p_sat = ps;
  return LBPC_OK;
}

LBPC_API lbpc_status lbpc_create(const lbpc_params* p, void* ws, size_t bytes, void* stream, lbpc_ctx** out) {
  if (!out) return LBPC_EINVAL;
  *out = nullptr;
  if (lbpc_check_params(p, nullptr, 0) != LBPC_OK) return LBPC_EINVAL;
  const Layout L = layout_of(p);
  if (!ws) return LBPC_EINVAL;
  if (((uintptr_t)ws & 255) != 0) return LBPC_EINVAL;
  if (bytes < L.total) return LBPC_ENOMEM;
  lbpc_ctx* c = (lbpc_ctx*)aligned_alloc(64, (sizeof(lbpc_ctx) + 63) / 64 * 64);
  if (!c) return LBPC_ENOMEM;
  memset(c, 0, sizeof(lbpc_ctx));
  c->p = *p;
  c->dp = make_dev_params(p);
  if (cudaGetDevice(&c->device) != cudaSuccess) {
    free(c);
    return LBPC_ECUDA;
  }
  c->stream = (cudaStream_t)stream;
  char* base = (char*)ws;
  for (int k = 0; k < 2; ++k) {
    c->buf.f[k] = base + L.f[k];
    c->buf.g[k] = base + L.g[k];
    c->buf.ref_f[k] = p->prec == LBPC_FP16DEV ? (float*)(base + L.ref_f[k]) : nullptr;
    c->buf.ref_g[k] = p->prec == LBPC_FP16DEV ? (float*)(base + L.ref_g[k]) : nullptr;
    c->buf.wall[k] = (double*)(base + L.wall[k]);
  }
  c->stage_bytes = 2 * (L.g[0] - L.f[0]);
  c->buf.phi_prev = base + L.phi;
  const size_t plane = align256((size_t)L.N * L.real);
  for (int k = 0; k < lbpc::split_nplanes(); ++k) c->buf.planes[k] = base + L.planes + k * plane;
  c->buf.partials = (double*)(base + L.partials);
  c->buf.scalars = (double*)(base + L.scalars);
  c->buf.status = (long long*)(base + L.status);
  c->cur = 0;
  c->step = 0;
  c->err = LBPC_OK;
  c->msg[0] = 0;
  c->buf.fused_tile = lbpc::kDefaultFusedTile;
  for (int k = 0; k < 2; ++k)
    if (lbpc::fused_tma_encode(&c->tma[k], p->prec, c->buf.fused_tile, c->buf.f[k], c->buf.g[k], c->buf.ref_f[k],
                               c->buf.ref_g[k], c->dp))
      c->buf.tma[k] = &c->tma[k];
  *out = c;
  return LBPC_OK;
}

static char* dead_half(lbpc_ctx* c) { return (char*)c->buf.f[c->cur ^ 1]; }

LBPC_API lbpc_status lbpc_init(lbpc_ctx* c, const double* rho, const double* T, const double* ux, const double* uy,
                               int on_device) {
  lbpc::TraceRange trace_("lbpc_init");
  if (!c) return LBPC_EINVAL;
  if (c->err != LBPC_OK) return LBPC_ESTATE;
  if (!rho || !T) return fail(c, LBPC_EINVAL, "lbpc_init: rho and T are required");
  DeviceGuard g(c->device);
  const size_t nb = (size_t)c->dp.N * sizeof(double);
  const double *d_rho = rho, *d_T = T, *d_ux = ux, *d_uy = uy;
  if (!on_device) {  // stage in the B half (the init kernel writes the A half)
    double* s = (double*)c->buf.f[1];
    CU(c, cudaMemcpyAsync(s, rho, nb, cudaMemcpyHostToDevice, c->stream), "lbpc_init H2D rho");
    CU(c, cudaMemcpyAsync(s + c->dp.N, T, nb, cudaMemcpyHostToDevice, c->stream), "lbpc_init H2D T");
    d_rho = s;
    d_T = s + c->dp.N;
    d_ux = d_uy = nullptr;
    if (ux) {
      CU(c, cudaMemcpyAsync(s + 2 * c->dp.N, ux, nb, cudaMemcpyHostToDevice, c->stream), "lbpc_init H2D ux");
      d_ux = s + 2 * c->dp.N;
    }
    if (uy) {
      CU(c, cudaMemcpyAsync(s + 3 * c->dp.N, uy, nb, cudaMemcpyHostToDevice, c->stream), "lbpc_init H2D uy");
      d_uy = s + 3 * c->dp.N;
    }
  }
  CU(c, cudaMemsetAsync(c->buf.status, 0, 8 * sizeof(long long), c->stream), "lbpc_init status reset");
  CU(c, lbpc::split_init(c->buf, c->dp, c->p.prec, d_rho, d_T, d_ux, d_uy, c->stream), "lbpc_init kernels");
  CU(c, cudaStreamSynchronize(c->stream), "lbpc_init sync");
  c->cur = 0;
  c->step = 0;
  c->initialised = 1;
  return LBPC_OK;
}

// The fused step's grid has one row of CTAs per tile row; the smallest tile is 8 rows high and a
// launch holds at most 65,535 rows of CTAs.
static bool fused_grid_fits(const lbpc_params& p) { return (p.ny + 7) / 8 <= 65535; }

static bool use_fused(const lbpc_ctx* c) {
  return c->path == LBPC_PATH_FUSED ||
         (c->path == LBPC_PATH_AUTO && c->p.prec != LBPC_FP64 && c->p.prec != LBPC_DF64 && fused_grid_fits(c->p));
}

static cudaError_t launch_step(lbpc_ctx* c, cudaEvent_t* ev) {
  return use_fused(c) ? lbpc::fused_step(c->buf, c->dp, c->p.prec, c->cur, c->step, c->stream, ev)
                      : lbpc::split_step(c->buf, c->dp, c->p.prec, c->cur, c->step, c->stream, ev);
}

static int step_kernel_count(const lbpc_ctx* c) {
  return use_fused(c) ? (c->dp.buoyancy == 1 ? 2 : 1) : lbpc::split_kernel_count(c->dp);
}

static const char* step_kernel_name(const lbpc_ctx* c, int k) {
  if (use_fused(c)) return k == 0 ? "k_fused" : (k == 1 ? "k_finish" : "");
  return lbpc::split_kernel_name(k);
}

LBPC_API lbpc_status lbpc_set_path(lbpc_ctx* c, int32_t path) {
  if (!c || path < LBPC_PATH_AUTO || path > LBPC_PATH_FUSED) return LBPC_EINVAL;
  if (path == LBPC_PATH_FUSED && !fused_grid_fits(c->p)) return LBPC_EINVAL;
  c->path = path;
  return LBPC_OK;
}

LBPC_API lbpc_status lbpc_set_fused_tile(lbpc_ctx* c, int32_t tile) {
  if (!c || tile < 0 || tile > 4) return LBPC_EINVAL;
  c->buf.fused_tile = tile;
  for (int k = 0; k < 2; ++k) {
    c->buf.tma[k] = nullptr;
    if (lbpc::fused_tma_encode(&c->tma[k], c->p.prec, tile, c->buf.f[k], c->buf.g[k], c->buf.ref_f[k], c->buf.ref_g[k],
                               c->dp))
      c->buf.tma[k] = &c->tma[k];
  }
  return LBPC_OK;
}

LBPC_API lbpc_status lbpc_step_async(lbpc_ctx* c, int64_t n) {
  lbpc::TraceRange trace_("lbpc_step_async");
  if (!c || n < 0) return LBPC_EINVAL;
  if (c->err != LBPC_OK) return LBPC_ESTATE;
  if (!c->initialised) return fail(c, LBPC_ESTATE, "lbpc_step before lbpc_init");
  DeviceGuard g(c->device);
  for (int64_t k = 0; k < n; ++k) {
    CU(c, launch_step(c, nullptr), "lbpc_step launch");
    c->cur ^= 1;
    ++c->step;
  }
  return LBPC_OK;
}

static lbpc_status check_status(lbpc_ctx* c) {
  long long st[5];
  CU(c, cudaMemcpyAsync(st, c->buf.status, sizeof st, cudaMemcpyDeviceToHost, c->stream), "status D2H");
  CU(c, cudaStreamSynchronize(c->stream), "status sync");
  if (st[0] != 0) {
    static const char* what[] = {"?", "rho <= 0", "rho >= 1/b (EOS pole)", "T <= 0", "psi^2 < 0", "non-finite value",
                                 "a bounded wait for a tile copy gave up"};
    char m[256];
    snprintf(m, sizeof m, "%s at step %lld, node (x=%lld, y=%lld): %s",
             st[4] == lbpc::ST_TIMEOUT ? "device timeout" : "non-physical state", st[1], st[2], st[3],
             what[(st[4] >= 1 && st[4] <= 6) ? st[4] : 0]);
    return fail(c, st[4] == lbpc::ST_TIMEOUT ? LBPC_ETIMEOUT : LBPC_ENONPHYS, m);
  }
  return LBPC_OK;
}

LBPC_API lbpc_status lbpc_check(lbpc_ctx* c) {
  if (!c) return LBPC_EINVAL;
  if (c->err != LBPC_OK) return c->err;
  DeviceGuard g(c->device);
  return check_status(c);
}

LBPC_API lbpc_status lbpc_step(lbpc_ctx* c, int64_t n) {
  lbpc_status s = lbpc_step_async(c, n);
  if (s != LBPC_OK) return s;
  DeviceGuard g(c->device);
  return check_status(c);
}

LBPC_API lbpc_status lbpc_step_timed(lbpc_ctx* c, float* kernel_ms, int32_t max_kernels, int32_t* n_kernels) {
  lbpc::TraceRange trace_("lbpc_step_timed");
  if (!c || (max_kernels > 0 && !kernel_ms)) return LBPC_EINVAL;
  if (c->err != LBPC_OK) return LBPC_ESTATE;
  if (!c->initialised) return fail(c, LBPC_ESTATE, "lbpc_step_timed before lbpc_init");
  DeviceGuard g(c->device);
  if (!c->have_events) {
    for (int k = 0; k < 8; ++k) CU(c, cudaEventCreate(&c->ev[k]), "lbpc_step_timed event create");
    c->have_events = 1;
  }
  const int nk = step_kernel_count(c);
  CU(c, launch_step(c, c->ev), "lbpc_step_timed launch");
  c->cur ^= 1;
  ++c->step;
  CU(c, cudaEventSynchronize(c->ev[nk]), "lbpc_step_timed sync");
  for (int k = 0; k < nk && k < max_kernels; ++k) {
    float ms = 0.f;
    CU(c, cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]), "lbpc_step_timed elapsed");
    kernel_ms[k] = ms;
  }
  if (n_kernels) *n_kernels = nk;
  return check_status(c);
}

LBPC_API const char* lbpc_kernel_name(const lbpc_ctx* c, int32_t k) {
  if (!c || k < 0 || k >= step_kernel_count(c)) return "";
  return step_kernel_name(c, k);
}

LBPC_API lbpc_status lbpc_fields(lbpc_ctx* c, double* rho, double* ux, double* uy, double* T, int on_device) {
  lbpc::TraceRange trace_("lbpc_fields");
  if (!c) return LBPC_EINVAL;
  if (!c->initialised) return LBPC_ESTATE;
  DeviceGuard g(c->device);
  const long long N = c->dp.N;
  const size_t nb = (size_t)N * sizeof(double);
  if (on_device) {
    CU(c, lbpc::split_fields(c->buf, c->dp, c->p.prec, c->cur, c->step, rho, ux, uy, T, c->stream), "lbpc_fields kernels");
    CU(c, cudaStreamSynchronize(c->stream), "lbpc_fields sync");
  } else {
    double* s = (double*)dead_half(c);
    double* d[4] = {rho ? s : nullptr, ux ? s + N : nullptr, uy ? s + 2 * N : nullptr, T ? s + 3 * N : nullptr};
    CU(c, lbpc::split_fields(c->buf, c->dp, c->p.prec, c->cur, c->step, d[0], d[1], d[2], d[3], c->stream), "lbpc_fields kernels");
    double* h[4] = {rho, ux, uy, T};
    for (int k = 0; k < 4; ++k)
      if (h[k]) CU(c, cudaMemcpyAsync(h[k], d[k], nb, cudaMemcpyDeviceToHost, c->stream), "lbpc_fields D2H");
    CU(c, cudaStreamSynchronize(c->stream), "lbpc_fields sync");
  }
  if (c->err == LBPC_OK) return check_status(c);
  return LBPC_OK;
}

// ---- checkpoint / resume ----
// Layout: a 512-byte header, then f and g of the current state (storage type, [9][N] each), the FP16
// reference planes of f and g (FP16 storage only), phi_prev ([N] of the arithmetic type) and the wall
// rows' force kept with f (FP64 [4][nx]).
namespace {
constexpr char kCkptMagic[8] = {'L', 'B', 'P', 'C', 'C', 'K', 'P', '1'};
constexpr uint32_t kCkptVersion = 2;  // 2: the wall-force section
constexpr size_t kCkptHeader = 512;
struct CkptHeader {
  char magic[8];
  uint32_t version, header_bytes;
  lbpc_params params;  // no padding inside the struct: compared bytewise on load
  int64_t step;
  double rho_ave;
  uint64_t pop_bytes, ref_bytes, phi_bytes, wall_bytes;
};
static_assert(sizeof(CkptHeader) <= kCkptHeader, "checkpoint header fits its slot");
static_assert(sizeof(lbpc_params) == 16 * 4 + 39 * 8, "lbpc_params has no padding");

void ckpt_sizes(const lbpc_ctx* c, size_t& pop, size_t& ref, size_t& phi, size_t& wall) {
  const Layout L = layout_of(&c->p);
  pop = 9 * (size_t)L.N * L.store;
  ref = c->p.prec == LBPC_FP16DEV ? (size_t)L.N * sizeof(float) : 0;
  phi = (size_t)L.N * L.real;
  wall = (size_t)lbpc::wall_doubles(c->p.nx) * sizeof(double);
}
}  // namespace

LBPC_API size_t lbpc_checkpoint_bytes(const lbpc_ctx* c) {
  if (!c) return 0;
  size_t pop, ref, phi, wall;
  ckpt_sizes(c, pop, ref, phi, wall);
  return kCkptHeader + 2 * pop + 2 * ref + phi + wall;
}

LBPC_API lbpc_status lbpc_save(lbpc_ctx* c, void* buf, size_t bytes, int on_device) {
  lbpc::TraceRange trace_("lbpc_save");
  if (!c || !buf) return LBPC_EINVAL;
  if (c->err != LBPC_OK) return LBPC_ESTATE;
  if (!c->initialised) return fail(c, LBPC_ESTATE, "lbpc_save before lbpc_init");
  if (bytes < lbpc_checkpoint_bytes(c)) return LBPC_EINVAL;
  DeviceGuard g(c->device);
  size_t pop, ref, phi, wall;
  ckpt_sizes(c, pop, ref, phi, wall);
  CkptHeader h{};
  memcpy(h.magic, kCkptMagic, sizeof h.magic);
  h.version = kCkptVersion;
  h.header_bytes = (uint32_t)kCkptHeader;
  h.params = c->p;
  h.step = c->step;
  h.pop_bytes = pop;
  h.ref_bytes = ref;
  h.phi_bytes = phi;
  h.wall_bytes = wall;
  CU(c, cudaMemcpyAsync(&h.rho_ave, c->buf.scalars, sizeof(double), cudaMemcpyDeviceToHost, c->stream),
     "lbpc_save rho_ave");
  CU(c, cudaStreamSynchronize(c->stream), "lbpc_save sync");
  unsigned char header[kCkptHeader] = {};
  memcpy(header, &h, sizeof h);
  unsigned char* dst = (unsigned char*)buf;
  const cudaMemcpyKind d2x = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CU(c, cudaMemcpyAsync(dst, header, kCkptHeader, on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost,
                        c->stream),
     "lbpc_save header");
  size_t off = kCkptHeader;
  CU(c, cudaMemcpyAsync(dst + off, c->buf.f[c->cur], pop, d2x, c->stream), "lbpc_save f");
  off += pop;
  CU(c, cudaMemcpyAsync(dst + off, c->buf.g[c->cur], pop, d2x, c->stream), "lbpc_save g");
  off += pop;
  if (ref) {
    CU(c, cudaMemcpyAsync(dst + off, c->buf.ref_f[c->cur], ref, d2x, c->stream), "lbpc_save ref_f");
    off += ref;
    CU(c, cudaMemcpyAsync(dst + off, c->buf.ref_g[c->cur], ref, d2x, c->stream), "lbpc_save ref_g");
    off += ref;
  }
  CU(c, cudaMemcpyAsync(dst + off, c->buf.phi_prev, phi, d2x, c->stream), "lbpc_save phi_prev");
  off += phi;
  CU(c, cudaMemcpyAsync(dst + off, c->buf.wall[c->cur], wall, d2x, c->stream), "lbpc_save wall");
  CU(c, cudaStreamSynchronize(c->stream), "lbpc_save sync");
  return LBPC_OK;
}

LBPC_API lbpc_status lbpc_load(lbpc_ctx* c, const void* buf, size_t bytes, int on_device) {
  lbpc::TraceRange trace_("lbpc_load");
  if (!c || !buf) return LBPC_EINVAL;
  if (c->err != LBPC_OK) return LBPC_ESTATE;
  if (bytes < lbpc_checkpoint_bytes(c)) return fail(c, LBPC_EINVAL, "lbpc_load: checkpoint smaller than expected");
  DeviceGuard g(c->device);
  const unsigned char* src = (const unsigned char*)buf;
  CkptHeader h{};
  if (on_device) {
    CU(c, cudaMemcpy(&h, src, sizeof h, cudaMemcpyDeviceToHost), "lbpc_load header");
  } else {
    memcpy(&h, src, sizeof h);
  }
  size_t pop, ref, phi, wall;
  ckpt_sizes(c, pop, ref, phi, wall);
  if (memcmp(h.magic, kCkptMagic, sizeof h.magic) != 0 || h.version != kCkptVersion || h.header_bytes != kCkptHeader)
    return fail(c, LBPC_EINVAL, "lbpc_load: not a liblbpc checkpoint");
  if (memcmp(&h.params, &c->p, sizeof(lbpc_params)) != 0)
    return fail(c, LBPC_EINVAL, "lbpc_load: the checkpoint was taken with other parameters");
  if (h.pop_bytes != pop || h.ref_bytes != ref || h.phi_bytes != phi || h.wall_bytes != wall || h.step < 0)
    return fail(c, LBPC_EINVAL, "lbpc_load: section sizes do not match");
  const cudaMemcpyKind x2d = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  size_t off = kCkptHeader;
  CU(c, cudaMemcpyAsync(c->buf.f[0], src + off, pop, x2d, c->stream), "lbpc_load f");
  off += pop;
  CU(c, cudaMemcpyAsync(c->buf.g[0], src + off, pop, x2d, c->stream), "lbpc_load g");
  off += pop;
  if (ref) {
    CU(c, cudaMemcpyAsync(c->buf.ref_f[0], src + off, ref, x2d, c->stream), "lbpc_load ref_f");
    off += ref;
    CU(c, cudaMemcpyAsync(c->buf.ref_g[0], src + off, ref, x2d, c->stream), "lbpc_load ref_g");
    off += ref;
  }
  CU(c, cudaMemcpyAsync(c->buf.phi_prev, src + off, phi, x2d, c->stream), "lbpc_load phi_prev");
  off += phi;
  CU(c, cudaMemcpyAsync(c->buf.wall[0], src + off, wall, x2d, c->stream), "lbpc_load wall");
  CU(c, cudaMemcpyAsync(c->buf.scalars, &h.rho_ave, sizeof(double), cudaMemcpyHostToDevice, c->stream),
     "lbpc_load rho_ave");
  CU(c, cudaMemsetAsync(c->buf.status, 0, 8 * sizeof(long long), c->stream), "lbpc_load status reset");
  CU(c, cudaStreamSynchronize(c->stream), "lbpc_load sync");
  c->cur = 0;
  c->step = h.step;
  c->initialised = 1;
  return LBPC_OK;
}

LBPC_API lbpc_status lbpc_sums(lbpc_ctx* c, double* mass, double* heat) {
  lbpc::TraceRange trace_("lbpc_sums");
  if (!c) return LBPC_EINVAL;
  if (!c->initialised) return LBPC_ESTATE;
  DeviceGuard g(c->device);
  double s[2];
  CU(c, lbpc::split_sums(c->buf, c->dp, c->p.prec, c->cur, c->stream), "lbpc_sums kernels");
  CU(c, cudaMemcpyAsync(s, c->buf.scalars + 1, sizeof s, cudaMemcpyDeviceToHost, c->stream), "lbpc_sums D2H");
  CU(c, cudaStreamSynchronize(c->stream), "lbpc_sums sync");
  if (mass) *mass = s[0];
  if (heat) *heat = s[1];
  return LBPC_OK;
}

LBPC_API lbpc_status lbpc_sums_async(lbpc_ctx* c, double* out, int on_device) {
  lbpc::TraceRange trace_("lbpc_sums_async");
  if (!c || !out) return LBPC_EINVAL;
  if (!c->initialised) return LBPC_ESTATE;
  DeviceGuard g(c->device);
  CU(c, lbpc::split_sums(c->buf, c->dp, c->p.prec, c->cur, c->stream), "lbpc_sums_async kernels");
  CU(c, cudaMemcpyAsync(out, c->buf.scalars + 1, 2 * sizeof(double),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream),
     "lbpc_sums_async copy");
  return LBPC_OK;
}

LBPC_API lbpc_status lbpc_populations(lbpc_ctx* c, double* f, double* g, int on_device) {
  lbpc::TraceRange trace_("lbpc_populations");
  if (!c) return LBPC_EINVAL;
  if (!c->initialised) return LBPC_ESTATE;
  DeviceGuard dg(c->device);
  const size_t nb = 9 * (size_t)c->dp.N * sizeof(double);
  double* outs[2] = {f, g};
  const size_t plane = (size_t)c->dp.N * sizeof(double);
  for (int which = 0; which < 2; ++which) {
    if (!outs[which]) continue;
    if (on_device) {
      CU(c, lbpc::split_export_pops(c->buf, c->dp, c->p.prec, c->cur, which, -1, outs[which], c->stream),
         "lbpc_populations kernel");
    } else if (c->stage_bytes >= nb) {  // all 9 planes through the dead half at once
      double* dst = (double*)dead_half(c);
      CU(c, lbpc::split_export_pops(c->buf, c->dp, c->p.prec, c->cur, which, -1, dst, c->stream),
         "lbpc_populations kernel");
      CU(c, cudaMemcpyAsync(outs[which], dst, nb, cudaMemcpyDeviceToHost, c->stream), "lbpc_populations D2H");
    } else {  // narrow storage: one plane at a time
      double* dst = (double*)dead_half(c);
      for (int a = 0; a < 9; ++a) {
        CU(c, lbpc::split_export_pops(c->buf, c->dp, c->p.prec, c->cur, which, a, dst, c->stream),
           "lbpc_populations kernel");
        CU(c, cudaMemcpyAsync(outs[which] + (size_t)a * c->dp.N, dst, plane, cudaMemcpyDeviceToHost, c->stream),
           "lbpc_populations D2H");
        CU(c, cudaStreamSynchronize(c->stream), "lbpc_populations sync");
      }
    }
    CU(c, cudaStreamSynchronize(c->stream), "lbpc_populations sync");
  }
  return LBPC_OK;
}

LBPC_API int64_t lbpc_step_count(const lbpc_ctx* c) { return c ? c->step : -1; }

LBPC_API const char* lbpc_last_error(const lbpc_ctx* c) { return c ? c->msg : "null context"; }

LBPC_API void lbpc_destroy(lbpc_ctx* c) {
  if (!c) return;
  if (c->have_events) {
    DeviceGuard g(c->device);
    for (int k = 0; k < 8; ++k) cudaEventDestroy(c->ev[k]);
  }
  free(c);
}
