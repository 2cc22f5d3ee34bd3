/*
 * lbpc.h - C ABI of liblbpc, the GB300 (sm_103a) implementation of the coupled lattice Boltzmann
 * time step for liquid-vapor phase change of Li, Zhou & Yan, "Improved thermal lattice Boltzmann
 * model for simulation of liquid-vapor phase change" (arXiv:1709.04400).
 *
 * One step on a 2D D2Q9 grid is: pseudopotential psi from the Peng-Robinson EOS at local (rho, T)
 * (Eq. 56), the neighbour-sum interaction force, the MRT density collide with forcing plus stream
 * (the flow model the paper takes from its Refs. [13,29]), and the improved thermal MRT step for T
 * (Eqs. 45-47 with the equilibria of Eq. 53, the source of Eq. 28 and the corrections of
 * Eqs. 54-55), with the moment and isotropic-gradient evaluations that feed it.
 *
 * Conventions for every function:
 *   - Lattice units: dt = dx = 1, c_s^2 = 1/3. Fields are row-major [ny][nx] (x fastest), FP64,
 *     whatever the storage precision of the populations.
 *   - Every function returns an lbpc_status; nothing throws across the ABI. The first error of a
 *     context is sticky: later calls that would advance or change the state return LBPC_ESTATE,
 *     while lbpc_fields, lbpc_sums, lbpc_populations and lbpc_last_error still work.
 *   - The caller owns every buffer passed in (the device workspace included); the library owns only
 *     the context struct, which lbpc_destroy frees. The library never allocates device memory.
 *   - "on_device" = 1: pointers are device pointers (any CUDA allocation of the current device);
 *     0: host pointers (pageable or pinned), copied through the context's stream.
 *   - All device work runs on the stream given to lbpc_create.
 */
#ifndef LBPC_H
#define LBPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBPC_VERSION 1

typedef struct lbpc_ctx lbpc_ctx; /* opaque */

typedef enum {
  LBPC_OK = 0,
  LBPC_EINVAL = 1,    /* invalid argument or parameter set */
  LBPC_ENOMEM = 2,    /* workspace smaller than lbpc_workspace_bytes() */
  LBPC_ECUDA = 3,     /* a CUDA runtime call failed; lbpc_last_error has its message */
  LBPC_ENONPHYS = 4,  /* rho <= 0, rho >= 1/b, T <= 0, psi^2 < 0 or non-finite; step, x, y reported */
  LBPC_ETIMEOUT = 5,  /* a bounded device-side wait gave up */
  LBPC_ESTATE = 6     /* the context holds an earlier error */
} lbpc_status;

/* Storage precision of the populations f, g and the arithmetic of the step.
 * LBPC_FP64: binary64 storage and arithmetic.
 * LBPC_FP32: binary32 storage and arithmetic.
 * LBPC_FP16DEV stores each post-collision population as binary16 of its deviation from the rest-state
 * equilibrium w_a * ref of the node that stored it, ref being that node's density (f) or
 * post-collision temperature (g), kept in FP32 planes beside the populations: 2 bytes per population
 * plus 4 per node and set, 96 B per node and step against 152 B for LBPC_FP32. Arithmetic is FP32.
 * LBPC_DF64: storage and arithmetic in double-word numbers, the unevaluated sum of two binary32
 * values (48-bit significand, relative precision about 3.6e-15, binary32 exponent range), 8 bytes per
 * value like LBPC_FP64. Every operation runs on the FP32 pipes; on GPUs whose binary64 rate is a
 * small fraction of the binary32 rate (GB300: 1/64) the step is several times faster than LBPC_FP64
 * and follows a binary64 evaluation of the same step to about 1e-12 over thousands of steps.
 * Inputs and outputs of the API are binary64 for every precision. */
typedef enum { LBPC_FP64 = 0, LBPC_FP32 = 1, LBPC_FP16DEV = 2, LBPC_DF64 = 3 } lbpc_prec;

/* Flow boundary of an edge. x edges must be periodic; y edges are both periodic or both not.
 * A non-periodic y edge is an on-node row closed by the Zou-He scheme (the paper applies Zou-He at
 * the solid surface, Sec. IV A, citing its Ref. [51]): LBPC_WALL = no-slip wall, LBPC_PRESSURE =
 * fixed density rho_bc with u_x = 0 (the open / fixed-pressure top). A wall sets the momentum of its
 * row to j = -F/2, F being the row's force of the previous step, so that the forcing scheme's
 * velocity v = (j + F/2)/rho vanishes there; with j = 0 a force on the wall row (the adsorption
 * force, buoyancy) would move fluid through the wall. The state therefore holds the wall rows' force
 * beside the populations. */
typedef enum { LBPC_PERIODIC = 0, LBPC_WALL = 1, LBPC_PRESSURE = 2 } lbpc_flow_bc;

/* Thermal boundary of an edge: LBPC_T_DIRICHLET holds T = T_bc on the edge row/column (the
 * constant-temperature boundaries of Sec. IV A and IV B). On a non-periodic y edge without a
 * Dirichlet T the unknown g populations bounce back (zero normal heat flux). */
typedef enum { LBPC_T_NONE = 0, LBPC_T_DIRICHLET = 1 } lbpc_thermal_bc;

/* Thermal conductivity: constant lambda (Sec. IV A) or lambda = rho c_V chi (Sec. IV A, B), for
 * which div(lambda grad T) = lambda lap T + grad lambda . grad T. */
typedef enum { LBPC_LAMBDA_CONST = 0, LBPC_LAMBDA_RHO_CV_CHI = 1 } lbpc_lambda_mode;

/* LBPC_IMPROVED: the paper's model (Eq. 53 equilibria, S0 = phi + 0.5 dt d_t phi, Eqs. 54-55).
 * LBPC_COMPROMISED: the comparison model of Sec. IV (Eq. 44 equilibria, S0 = phi, no corrections).
 * LBPC_GONG_CHENG: the model the paper improves on (Eqs. 11-14): BGK with the second-order
 * equilibrium of Eq. 14, tau_g = lambda/(rho c_s^2 c_V) + 1/2 (Sec. IV A) and the source w_a phi of
 * Eq. 13; s_g is not used. */
typedef enum { LBPC_IMPROVED = 0, LBPC_COMPROMISED = 1, LBPC_GONG_CHENG = 2 } lbpc_thermal_model;

/* Edge order in the arrays below: 0 = x-, 1 = x+, 2 = y- (bottom, y = 0), 3 = y+ (top, y = ny-1). */
typedef struct {
  int32_t nx, ny;          /* grid; nx >= 2, ny >= 2 (ny >= 3 with non-periodic y) */
  int32_t prec;            /* lbpc_prec */
  int32_t model;           /* lbpc_thermal_model */
  int32_t lambda_mode;     /* lbpc_lambda_mode */
  int32_t buoyancy;        /* 0: no body force. 1: F_b = (rho - rho_ave) g with rho_ave the domain mean of the
                              previous step (Sec. IV B; its total vanishes in a closed or periodic domain).
                              2: F_b = (rho - rho_bc[3]) g, the reference being the density held on a
                              LBPC_PRESSURE y+ edge: under an open top the vapour there is force-free, where
                              mode 1 accelerates it out without bound. Other values: LBPC_EINVAL */
  int32_t flow_bc[4];      /* lbpc_flow_bc per edge */
  int32_t t_bc[4];         /* lbpc_thermal_bc per edge */
  int32_t strip_x0, strip_x1; /* heated strip [x0, x1) on the y- row at T_strip (needs t_bc[2]); x0 = x1: none */
  double a, b, R, omega;   /* Peng-Robinson EOS, Eq. 56 (paper: 3/49, 2/21, 1, 0.344) */
  double G;                /* interaction strength of the pseudopotential force (reading: -1) */
  double s_f[9];           /* flow MRT rates, moments (rho,e,eps,jx,qx,jy,qy,pxx,pxy); s_f[7]=s_f[8]=1/(3 nu+1/2) */
  double s_g[9];           /* thermal MRT rates (Eq. 43); k = (1/s_g[3] - 1/2)/3 (Eq. 41); s_g[5] = s_g[3] */
  double sigma;            /* mechanical-stability coefficient of the flow forcing (reading: 0.1) */
  double lambda;           /* constant thermal conductivity (LBPC_LAMBDA_CONST) */
  double chi;              /* thermal diffusivity for lambda = rho c_V chi */
  double cV;               /* specific heat at constant volume */
  double gx, gy;           /* gravitational acceleration g (Sec. IV B uses g = (0, -g)) */
  double rho_bc[4];        /* density held on LBPC_PRESSURE edges */
  double T_bc[4];          /* temperature held on LBPC_T_DIRICHLET edges */
  double T_strip;          /* temperature of the heated strip */
  double G_wall;           /* fluid-solid strength: F_ads = -G_wall psi(x) sum_a w_a psi(x) s(x+e_a) e_a at
                              the y- wall (G_wall < 0 wets); a y+ wall is a neutral lid */
} lbpc_params;

/* Library version (LBPC_VERSION). */
int32_t lbpc_version(void);

/* Validate a parameter set. Returns LBPC_OK or LBPC_EINVAL and writes a reason into msg
 * (NUL-terminated, at most msg_len bytes) when msg is not NULL. No device work. */
lbpc_status lbpc_check_params(const lbpc_params* p, char* msg, size_t msg_len);

/* Bytes of device workspace a context with these parameters needs (0 if the parameters are
 * invalid). The caller allocates it (any device allocation aligned to 256 bytes). */
size_t lbpc_workspace_bytes(const lbpc_params* p);

/* Critical temperature and pressure of the Peng-Robinson EOS: T_c = 0.0778 a / (0.45724 b R),
 * p_c = 0.0778 R T_c / b (both follow from the definitions of a and b after Eq. 56). Host only. */
lbpc_status lbpc_eos_critical(const lbpc_params* p, double* Tc, double* pc);

/* Liquid-vapor coexistence of Eq. 56 at temperature T < T_c (equal pressure and equal fugacity):
 * writes rho_v < rho_l and the saturation pressure. Host only; LBPC_EINVAL if T >= T_c. */
lbpc_status lbpc_coexistence(const lbpc_params* p, double T, double* rho_v, double* rho_l, double* p_sat);

/* Create a context on the current CUDA device. d_workspace: caller-owned device buffer of at least
 * lbpc_workspace_bytes(p) bytes, borrowed until lbpc_destroy. stream: a cudaStream_t (NULL = the
 * legacy default stream). The populations are undefined until lbpc_init. */
lbpc_status lbpc_create(const lbpc_params* p, void* d_workspace, size_t bytes, void* stream, lbpc_ctx** out);

/* Set the state to equilibrium populations f = M^{-1} m_eq(rho, u), g = M^{-1} m_eq(T, u), closed
 * once by the boundary step, and reset the step counter. The thermal equilibrium is Eq. 53 for the
 * improved model (Eq. 44 for the compromised one; the moments of Eq. 14 for Gong-Cheng); M is the
 * MRT transform of Eqs. 42-43; the flow equilibrium is that of the delegated flow model (Sec. III B,
 * Refs. [13,29]). The first step takes phi(t - dt) = phi(t) in Eq. 46. rho, T: [ny][nx] FP64, host
 * memory, or device memory when on_device is nonzero (required, owned by the caller); ux, uy: [ny][nx]
 * FP64 or NULL for zero. LBPC_EINVAL for a null rho or T, LBPC_ESTATE after an earlier error; a start
 * outside the EOS range is reported by the first step. Synchronises the stream. */
lbpc_status lbpc_init(lbpc_ctx* c, const double* rho, const double* T, const double* ux, const double* uy,
                      int on_device);

/* Advance n >= 0 time steps and check the device status word once at the end (synchronises the
 * stream). One step is the paper's coupled update (Sec. III B, the model summary after Eq. 55): the
 * pull-stream of Eq. 47 with the boundary closures, the moments, the EOS of Eq. 56 and the
 * pseudopotential, the interaction, adsorption and buoyancy forces, the isotropic gradients, the source
 * of Eq. 28 with S0 of Eq. 46, the flow MRT collision with forcing and the thermal MRT collision of
 * Eqs. 45 and 53-55. Returns LBPC_ENONPHYS with step, x, y in lbpc_last_error if a node left the
 * physical range of the EOS during these steps; LBPC_ESTATE before lbpc_init or after an error. */
lbpc_status lbpc_step(lbpc_ctx* c, int64_t n);

/* Enqueue n time steps on the stream and return without synchronising or checking the device
 * status; the next lbpc_step / lbpc_fields / lbpc_sums / lbpc_check reports any error. */
lbpc_status lbpc_step_async(lbpc_ctx* c, int64_t n);

/* Advance exactly one time step with a CUDA event recorded on the context's stream before the first
 * kernel and after each kernel of the step; synchronise and write the duration of each kernel launch
 * in milliseconds to kernel_ms[0 .. *n_kernels) (at most max_kernels entries). lbpc_kernel_name
 * names them. Used to time the step's kernels live inside a benchmark. */
lbpc_status lbpc_step_timed(lbpc_ctx* c, float* kernel_ms, int32_t max_kernels, int32_t* n_kernels);

/* Name of kernel k of the step as lbpc_step_timed orders them ("" if k is out of range). */
const char* lbpc_kernel_name(const lbpc_ctx* c, int32_t k);

/* Kernel organisation of lbpc_step. LBPC_PATH_SPLIT: three node-parallel kernels per step with
 * scratch planes (each EOS evaluated once per node; the faster choice when FP64 arithmetic bounds
 * the step). LBPC_PATH_FUSED: one kernel per step over shared-memory tiles (populations read once
 * and written once; the faster choice when HBM bounds the step). LBPC_PATH_AUTO (default): split
 * for LBPC_FP64 and LBPC_DF64, fused for LBPC_FP32 and LBPC_FP16DEV. Both compute the same step.
 * The fused step launches one row of CTAs per 8 grid rows, and a launch has at most 65,535 rows of
 * CTAs: for ny > 524,280, LBPC_PATH_AUTO takes the split step and LBPC_PATH_FUSED returns
 * LBPC_EINVAL. */
typedef enum { LBPC_PATH_AUTO = 0, LBPC_PATH_SPLIT = 1, LBPC_PATH_FUSED = 2 } lbpc_path;
lbpc_status lbpc_set_path(lbpc_ctx* c, int32_t path);

/* Tile configuration of the fused step (LBPC_FP32 and LBPC_FP16DEV): 0 = 32 x 16 tiles, one node per
 * thread; 1 = 32 x 8, one node per thread (smaller shared-memory footprint, four CTAs per SM, more halo
 * recomputation); 2 = 32 x 16, two nodes per thread; 3 = 32 x 32, two nodes per thread (less halo
 * recomputation per node); 4 = 32 x 8 in persistent CTAs that take tiles in order and start each next
 * tile's staging copy while they finish the current tile (default). Where the rows are not 16-byte
 * multiples (no staging), 4 runs as 1. All compute the same step. LBPC_EINVAL outside 0..4. */
lbpc_status lbpc_set_fused_tile(lbpc_ctx* c, int32_t tile);

/* Synchronise the stream and check the device status word. */
lbpc_status lbpc_check(lbpc_ctx* c);

/* Macroscopic fields of the current state: rho = sum f, u = (sum e f + F/2)/rho (F as the next step
 * would use it), T = sum g. Any pointer may be NULL. [ny][nx] FP64. Synchronises the stream. */
lbpc_status lbpc_fields(lbpc_ctx* c, double* rho, double* ux, double* uy, double* T, int on_device);

/* Domain sums of rho (mass) and T (heat content) of the current state, accumulated in FP64 in a
 * fixed order. Synchronises the stream. */
lbpc_status lbpc_sums(lbpc_ctx* c, double* mass, double* heat);

/* The same sums without waiting: enqueues their kernels and a copy of {mass, heat} (two doubles) into
 * out on the context's stream and returns. out is pinned host memory (on_device = 0; pageable memory
 * also works, with a synchronous copy) or device memory (on_device = 1), owned by the caller and valid
 * until the stream has passed the copy (lbpc_check, or a synchronisation of the stream). A per-step
 * read of the result that keeps the stream busy. Returns LBPC_EINVAL for a null pointer,
 * LBPC_ESTATE before lbpc_init, LBPC_ECUDA if a launch fails; device-side errors surface at the next
 * lbpc_check / lbpc_step. */
lbpc_status lbpc_sums_async(lbpc_ctx* c, double* out, int on_device);

/* Checkpoint / resume. The paper has no counterpart; this is plumbing for long runs and for a
 * service that moves or pre-empts simulations.
 *
 * A checkpoint is the context's whole state in raw form:
 *   - a 512-byte header holding, in this order and without gaps: the 8 bytes "LBPCCKP1", the format
 *     version (uint32, 2), the header size (uint32, 512), the lbpc_params, the step counter (int64),
 *     the lagged rho_ave (double) and the byte sizes of the four sections below (uint64 each:
 *     populations of one set, reference planes of one set, phi, wall forces); the rest is zero;
 *   - the current post-collision populations f and g in the storage type, plus the FP16 reference
 *     planes for LBPC_FP16DEV;
 *   - phi of the previous step, in the arithmetic type;
 *   - the wall rows' force of the previous step (binary64 [4][nx]), which the next wall closure uses.
 * Stepping a context restored from a checkpoint taken after k steps reproduces, bit for bit, the
 * steps after k of an uninterrupted run with the same parameters and precision.
 *
 * lbpc_checkpoint_bytes: size of a checkpoint of this context (0 for a null context).
 * lbpc_save: writes it into buf (host memory, or device memory when on_device is nonzero), which is
 *   at least lbpc_checkpoint_bytes long and owned by the caller. The context must be initialised
 *   and free of errors (LBPC_ESTATE otherwise). LBPC_EINVAL if buf is too small. Synchronises the
 *   stream.
 * lbpc_load: replaces the state of a context created with the same lbpc_params (compared byte for
 *   byte; LBPC_EINVAL otherwise, and for a buffer that is not a checkpoint). The context need not
 *   be initialised. Clears the non-physical status. Synchronises the stream. */
size_t lbpc_checkpoint_bytes(const lbpc_ctx* c);
lbpc_status lbpc_save(lbpc_ctx* c, void* buf, size_t bytes, int on_device);
lbpc_status lbpc_load(lbpc_ctx* c, const void* buf, size_t bytes, int on_device);

/* Raw populations of the current state in post-stream, post-boundary form: f, g are [9][ny][nx]
 * FP64 (D2Q9 order e0=(0,0), e1=(1,0), e2=(0,1), e3=(-1,0), e4=(0,-1), e5=(1,1), e6=(-1,1),
 * e7=(-1,-1), e8=(1,-1)). Either pointer may be NULL. Synchronises the stream. */
lbpc_status lbpc_populations(lbpc_ctx* c, double* f, double* g, int on_device);

/* Number of time steps taken since lbpc_init. */
int64_t lbpc_step_count(const lbpc_ctx* c);

/* Message of the last error of the context ("" if none). Valid until the next call on c. */
const char* lbpc_last_error(const lbpc_ctx* c);

/* Free the context (not the workspace, not the stream). NULL is allowed. */
void lbpc_destroy(lbpc_ctx* c);

/* ------------------------------------------------------------------------------------------------
 * Batches: many independent simulations of uneven size advancing together.
 *
 * The per-node arithmetic is the fused step's. A step is a few per-tile launches, one CTA per tile,
 * each holding up to lbpc_batch_per_tile_capacity instances in its kernel parameters (the default),
 * or one launch whose CTAs walk a device-resident work list of (instance, tile) entries (see
 * lbpc_batch_set_config). Steps are replayed through captured CUDA graphs in chunks when the batch
 * has a non-default stream. Instances can join and leave between calls. Their parameters,
 * boundaries, sizes and step counts are their own, and an instance's result does not depend on
 * what else is in the batch. All instances of a batch share one storage precision.
 *
 * The batch takes one caller-owned device arena. The library carves every instance's state out of it
 * with a first-fit allocator and allocates no device memory of its own.
 * ------------------------------------------------------------------------------------------------ */
typedef struct lbpc_batch lbpc_batch; /* opaque */

/* Arena bytes one instance with these parameters takes (0 if the parameters are invalid). */
size_t lbpc_batch_instance_bytes(const lbpc_params* p);

/* Create an empty batch of at most max_instances instances in storage precision prec (LBPC_FP64,
 * LBPC_FP32 or LBPC_FP16DEV; LBPC_DF64 returns LBPC_EINVAL) over the caller's arena (256-byte
 * aligned, bytes long). Fixed descriptors take a small part of the arena. The initial configuration
 * is 32 x 8 tiles in per-tile launches (variant 0, 0 CTAs per SM; see lbpc_batch_set_config). */
lbpc_status lbpc_batch_create(int32_t prec, int32_t max_instances, void* d_arena, size_t bytes, void* stream,
                              lbpc_batch** out);

/* Add an instance started from the equilibrium of rho, T ([ny][nx] FP64, host or device), like
 * lbpc_init. Writes its id. LBPC_ENOMEM when the arena or the slots are full; LBPC_EINVAL when
 * 9 nx ny >= 2^31 (the step kernel forms population indices in 32 bits). Synchronises. */
lbpc_status lbpc_batch_add(lbpc_batch* b, const lbpc_params* p, const double* rho, const double* T, int on_device,
                           int32_t* id);

/* Remove an instance and return its memory to the arena. Synchronises. */
lbpc_status lbpc_batch_remove(lbpc_batch* b, int32_t id);

/* Enqueue n steps of every instance; does not synchronise (lbpc_batch_check reports errors). */
lbpc_status lbpc_batch_step(lbpc_batch* b, int64_t n);

/* Synchronise and check every instance's status word; LBPC_ENONPHYS names the first failed id. */
lbpc_status lbpc_batch_check(lbpc_batch* b, int32_t* failed_id);

/* Fields and domain sums of one instance, as lbpc_fields and lbpc_sums (scratch for the fields comes
 * from the arena for the duration of the call). Synchronise. */
lbpc_status lbpc_batch_fields(lbpc_batch* b, int32_t id, double* rho, double* ux, double* uy, double* T, int on_device);
lbpc_status lbpc_batch_sums(lbpc_batch* b, int32_t id, double* mass, double* heat);

/* Steps taken by instance id (-1 if no such instance). */
int64_t lbpc_batch_step_count(const lbpc_batch* b, int32_t id);

/* Step-kernel variant and CTAs launched per SM. Variants: 0 = 32x8, 1 = 32x16, 2 = 64x8 tiles with one
 * node per thread; 3 = 32x16, 4 = 64x16, 5 = 32x32 tiles with two nodes per thread.
 * ctas_per_sm >= 1: one launch per step of the work-list kernel, whose CTAs walk the device work list
 * from their index in steps of the grid size. Up to the residency limit of the variant, every CTA is
 * resident (a persistent grid). Above it, up to 64 times that limit, further CTAs start as earlier
 * ones finish, so the hardware balances tiles of uneven cost. A value above that returns LBPC_EINVAL.
 * ctas_per_sm = 0: per-tile launches. A step is a sequence of launches with one CTA per tile, each over
 * up to lbpc_batch_per_tile_capacity instances held in its kernel parameters; each launch may start
 * while the previous one drains. A change of instances then captures the step graphs again.
 * A negative value returns LBPC_EINVAL. */
lbpc_status lbpc_batch_set_config(lbpc_batch* b, int32_t variant, int32_t ctas_per_sm);

/* Instances one per-tile launch holds for storage precision prec (0 for a precision a batch does not
 * take). */
int32_t lbpc_batch_per_tile_capacity(int32_t prec);
lbpc_status lbpc_batch_config(const lbpc_batch* b, int32_t* tile_x, int32_t* tile_y, int32_t* ctas_per_sm,
                              int32_t* graph_chunk);

/* Time every variant (tile shape and nodes per thread) with per-tile launches, with the residency
 * limit of CTAs per SM and with 16, 32 and 64 times that limit on the batch's own instances, and keep
 * the fastest. Every configuration computes the same step, so tuning advances the batch by real steps:
 * per candidate, one graph chunk of warm-up (which captures its graph), then steps_per_candidate
 * rounded up to whole graph chunks, timed. */
lbpc_status lbpc_batch_autotune(lbpc_batch* b, int32_t steps_per_candidate, int32_t* best_variant, int32_t* best_ctas,
                                float* best_ms_per_step);

/* Free bytes left in the arena, the last error message, and teardown (the arena stays the caller's). */
size_t lbpc_batch_free_bytes(const lbpc_batch* b);
const char* lbpc_batch_last_error(const lbpc_batch* b);
void lbpc_batch_destroy(lbpc_batch* b);

/* ------------------------------------------------------------------------------------------------
 * FMA throughput of the current device: the measured denominator of the roofline of ALU-bound kernels
 * (the binary64 step is bound by the FP64 pipe on this GPU). The paper has no counterpart; this is a
 * measurement aid, not part of the method.
 *
 *   prec        LBPC_FP64 (binary64 FMA) or LBPC_FP32 (binary32 FMA)
 *   stream      cudaStream_t the probe runs on; the call synchronises it
 *   flop_per_s  receives 2 x the FMAs per second of one timed launch (after one warm-up launch) of a
 *               probe kernel whose threads each run 8 independent FMA chains, on every SM with as many
 *               CTAs as can be resident (about 30 ms in binary64, 20 ms in binary32)
 * Allocates no device memory. Returns LBPC_EINVAL for another prec or a null pointer, LBPC_ECUDA if a
 * launch fails. */
lbpc_status lbpc_fma_rate(int32_t prec, void* stream, double* flop_per_s);

/* ------------------------------------------------------------------------------------------------
 * One time step without any device allocation.
 *
 * Some callers cannot allocate device memory at all: an application whose device memory is handed
 * out only by its own pool allocator, code that runs where cudaMalloc is not permitted, or a host
 * program with no allocator of its own. lbpc_create needs a caller-allocated workspace that holds
 * scratch planes besides the state. lbpc_step_static instead takes only the state (inputs and outputs)
 * from the caller and keeps its scratch in a fixed static device array of the library. That array
 * is sized for at most LBPC_STATIC_MAX_NODES nodes (256 x 256), about 6 MiB, and every GPU that loads
 * the library holds it until the process exits. The paper has no counterpart; this is plumbing.
 *
 * It runs the same kernels as lbpc_step and lbpc_step_async, with the split organisation.
 *
 *   p         parameters, as for lbpc_create, with prec LBPC_FP64, LBPC_FP32 or LBPC_DF64; nx * ny must not
 *             exceed LBPC_STATIC_MAX_NODES (LBPC_ENOMEM otherwise, before any device work)
 *   f_in,g_in post-collision populations of the previous step, device, [9][ny][nx] of the storage type
 *             (lbpc_params.prec), D2Q9 order as for lbpc_populations; slot a of node x holds the value
 *             that node x + e_a receives when it streams. A context's state has this form.
 *   f_out,g_out  device buffers of the same size for the new post-collision populations; they must
 *             not alias the inputs
 *   wall_in   device [4][nx] doubles: the force on the wall rows (y- Fx, y- Fy, y+ Fx, y+ Fy) of the
 *             step that wrote f_in, zeros before the first step; entries of a non-wall edge are unused.
 *             Required when a y edge is LBPC_WALL, else it may be NULL
 *   wall_out  device [4][nx] doubles for this step's wall-row force (the next call's wall_in); it
 *             must not alias wall_in. Required and ignored as wall_in
 *   phi_prev  device [ny][nx] of the arithmetic type: phi of the previous step in, this step's out
 *             (ignored on input when step == 0)
 *   rho_ave   device pointer to one double: the previous step's domain mean of rho in, this step's
 *             out; used and updated only with buoyancy 1 (may be NULL otherwise)
 *   step      index of this step (0 = first step after the equilibrium start)
 *   stream    cudaStream_t the work runs on; the call synchronises it before returning
 * Returns LBPC_OK, LBPC_ENONPHYS if a node left the EOS range, LBPC_EINVAL, LBPC_ENOMEM or
 * LBPC_ECUDA.
 *
 * The call allocates nothing itself: no cudaMalloc, no cudaFree, no allocating library routine. Every
 * call looks up the device address of the static array in the device context that is current
 * (cudaGetSymbolAddress; an address is never carried over, so a device reset is harmless). Under CUDA's
 * default lazy module loading the array is placed in device memory when the library's module is
 * first used in a context, which can be the first lbpc_step_static call on that device: that first
 * call may therefore need about 6 MiB of free device memory, and it should come before any stream
 * capture. Later calls need no device memory at all. Every call shares the one array, which keeps
 * the last call's contents (the status word is cleared at the start of each call); calls that overlap
 * on the GPU, from several threads or streams, race on it. */
#define LBPC_STATIC_MAX_NODES (256 * 256)
lbpc_status lbpc_step_static(const lbpc_params* p, const void* f_in, const void* g_in, void* f_out, void* g_out,
                             const double* wall_in, double* wall_out, void* phi_prev, double* rho_ave, int64_t step,
                             void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LBPC_H */
