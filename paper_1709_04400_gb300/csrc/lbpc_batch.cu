// Host side of the batched step: many independent simulations of uneven size advance together, either
// as per-tile launches that hold the instances in their parameters (lbpc_batch_tiles.cu) or as one
// work-list launch per step (lbpc_batch_kernels.cu). The batch carves every instance's state out of one
// caller-owned device arena with a first-fit allocator, keeps the instance descriptors and a tile work
// list on the device, replays the steps through captured CUDA graphs, and picks its tile shape and
// launch form by timing.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <memory>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lbpc.h"
#include "lbpc_internal.h"

#define LBPC_API extern "C" __attribute__((visibility("default")))

namespace lbpc {
DevParams make_dev_params_public(const lbpc_params* p);
}

namespace {

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// First-fit allocator over [0, size) of the arena, 256-byte granules.
class Arena {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    size_ = size;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = a256(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes, start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = a256(bytes);
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {  // merge with the next block
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {  // merge with the previous block
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t free_bytes() const {
    size_t s = 0;
    for (auto& kv : free_) s += kv.second;
    return s;
  }
  size_t largest() const {
    size_t s = 0;
    for (auto& kv : free_) s = std::max(s, kv.second);
    return s;
  }

 private:
  std::map<size_t, size_t> free_;
  size_t size_ = 0;
};

struct HostInst {
  bool used = false;
  lbpc_params p{};
  lbpc::DevParams dp{};
  long long N = 0;
  size_t off = 0, bytes = 0;  // arena block of the instance
  size_t f[2], g[2], rf[2], rg[2], wall[2], phi, partials, scalars;
  size_t npartials = 0;
  long long step = 0;
  int cur = 0;
};

size_t store_bytes(int prec) { return prec == LBPC_FP64 ? 8 : (prec == LBPC_FP32 ? 4 : 2); }
size_t real_bytes(int prec) { return prec == LBPC_FP64 ? 8 : 4; }

// Lay out one instance inside a block starting at 0; returns the block size.
size_t layout_instance(const lbpc_params* p, HostInst* h) {
  const long long N = (long long)p->nx * p->ny;
  const size_t sb = store_bytes(p->prec), rb = real_bytes(p->prec);
  const size_t pop = a256(9 * (size_t)N * sb);
  size_t off = 0;
  // f0 g0 f1 g1 contiguous so the dead half can stage FP64 transfers
  for (int k = 0; k < 2; ++k) {
    h->f[k] = off; off += pop;
    h->g[k] = off; off += pop;
  }
  const size_t ref = p->prec == LBPC_FP16DEV ? a256((size_t)N * 4) : 0;
  for (int k = 0; k < 2; ++k) {
    h->rf[k] = off; off += ref;
    h->rg[k] = off; off += ref;
  }
  for (int k = 0; k < 2; ++k) {  // wall-row forces kept with f for the next step's wall closure
    h->wall[k] = off; off += a256((size_t)lbpc::wall_doubles(p->nx) * sizeof(double));
  }
  h->phi = off; off += a256((size_t)N * rb);
  h->npartials = std::max(lbpc::fused_max_tiles(p->nx, p->ny), 2 * (size_t)((N + lbpc::split_block() - 1) / lbpc::split_block()));
  h->partials = off; off += a256(h->npartials * sizeof(double));
  h->scalars = off; off += a256(8 * sizeof(double));
  return off;
}

}  // namespace

struct lbpc_batch {
  int prec;
  int max_inst;
  int device;
  cudaStream_t stream;
  char* base;
  size_t bytes;
  Arena arena;
  size_t meta_off, insts_off, status_off;  // reserved at creation
  size_t tiles_off = 0, tiles_cap = 0;     // work list block (grows)
  std::vector<HostInst> inst;
  size_t inst_struct;  // sizeof(BatchInst<S>)
  int variant = 0;     // tile shape (32 x 8)
  int ctas = 0;        // CTAs launched per SM by the work-list kernel; 0: per-tile launches
  int chunk = 16;      // steps per captured graph (even: a replay leaves every buffer parity as it was)
  // Captured graphs of `chunk` steps. The work-list kernel reads everything per instance from device
  // memory, so one graph serves every step parity and instance set ([0]). Per-tile launches carry
  // each instance's buffers for the parity of their step in their parameters: one graph per parity of
  // the steps taken, captured again when the instances change.
  struct GraphSlot {
    cudaGraphExec_t exec = nullptr;
    int variant = -1, ctas = -1, ninst = -1;
    long long gen = -1;
  } graphs[2];
  long long gen = 0;   // bumped by every rebuild (instances or configuration changed)
  int phase = 0;       // parity of the steps taken since creation
  bool dirty = true;   // work list needs a rebuild
  lbpc_status err = LBPC_OK;
  char msg[512] = {0};
};

namespace {

lbpc_status bfail(lbpc_batch* b, lbpc_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(b->msg, sizeof b->msg, fmt, ap);
  va_end(ap);
  return s;
}

#define BCU(b, call, where)                                                                          \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) {                                                                         \
      b->err = LBPC_ECUDA;                                                                           \
      return bfail(b, LBPC_ECUDA, "%s: %s (%s)", where, cudaGetErrorName(e_), cudaGetErrorString(e_)); \
    }                                                                                                \
  } while (0)

struct DevGuard {
  int old = -1;
  explicit DevGuard(int dev) {
    if (cudaGetDevice(&old) == cudaSuccess && old != dev) cudaSetDevice(dev);
    else old = -1;
  }
  ~DevGuard() {
    if (old >= 0) cudaSetDevice(old);
  }
};

size_t inst_struct_bytes(int prec) {
  return prec == LBPC_FP64 ? sizeof(lbpc::BatchInst<double>)
                           : (prec == LBPC_FP32 ? sizeof(lbpc::BatchInst<float>) : sizeof(lbpc::BatchInst<__half>));
}

// Device descriptor of instance k as raw bytes (the layout of BatchInst<S> for the batch's S).
template <class S> void fill_desc(lbpc_batch* b, int k, std::vector<char>& out) {
  lbpc::BatchInst<S> d{};
  const HostInst& h = b->inst[k];
  if (h.used) {
    char* base = b->base + h.off;
    d.P = h.dp;
    for (int j = 0; j < 2; ++j) {
      d.f[j] = lbpc::PopBuf<S>{(S*)(base + h.f[j]), b->prec == LBPC_FP16DEV ? (float*)(base + h.rf[j]) : nullptr,
                               (double*)(base + h.wall[j])};
      d.g[j] = lbpc::PopBuf<S>{(S*)(base + h.g[j]), b->prec == LBPC_FP16DEV ? (float*)(base + h.rg[j]) : nullptr};
    }
    d.phi_prev = base + h.phi;
    d.scalars = (double*)(base + h.scalars);
    d.partials = (double*)(base + h.partials);
    d.step = h.step;
    d.cur = h.cur;
    d.active = 1;
    int tx, ty;
    lbpc::batch_tile_shape(b->variant, tx, ty);
    d.ntiles = ((h.dp.nx + tx - 1) / tx) * ((h.dp.ny + ty - 1) / ty);
  }
  d.status = (long long*)(b->base + b->status_off) + 8 * k;
  out.resize(sizeof d);
  memcpy(out.data(), &d, sizeof d);
}

void desc_bytes(lbpc_batch* b, int k, std::vector<char>& out) {
  if (b->prec == LBPC_FP64) fill_desc<double>(b, k, out);
  else if (b->prec == LBPC_FP32) fill_desc<float>(b, k, out);
  else fill_desc<__half>(b, k, out);
}

lbpc_status upload_desc(lbpc_batch* b, int k) {
  std::vector<char> d;
  desc_bytes(b, k, d);
  BCU(b, cudaMemcpyAsync(b->base + b->insts_off + (size_t)k * b->inst_struct, d.data(), d.size(), cudaMemcpyHostToDevice,
                         b->stream),
      "batch descriptor upload");
  // pageable source: the copy is staged before the call returns, so d may go out of scope
  return LBPC_OK;
}

// Rebuild the work list (all tiles of every active instance, instance-major) and the meta block.
lbpc_status rebuild(lbpc_batch* b) {
  int tx, ty;
  lbpc::batch_tile_shape(b->variant, tx, ty);
  std::vector<lbpc::BatchTile> tiles;
  for (int k = 0; k < (int)b->inst.size(); ++k) {
    const HostInst& h = b->inst[k];
    if (!h.used) continue;
    int slot = 0;
    for (int y0 = 0; y0 < h.dp.ny; y0 += ty)
      for (int x0 = 0; x0 < h.dp.nx; x0 += tx) tiles.push_back(lbpc::BatchTile{k, x0, y0, slot++});
  }
  const size_t need = std::max<size_t>(tiles.size(), 1) * sizeof(lbpc::BatchTile);
  if (need > b->tiles_cap) {
    BCU(b, cudaStreamSynchronize(b->stream), "batch work list sync");  // the old list may still be read
    if (b->tiles_cap) b->arena.release(b->tiles_off, b->tiles_cap);
    const size_t cap = a256(need + need / 2);
    if (!b->arena.alloc(cap, &b->tiles_off)) {
      b->tiles_cap = 0;
      return bfail(b, LBPC_ENOMEM, "arena full: no room for a work list of %zu tiles", tiles.size());
    }
    b->tiles_cap = cap;
  }
  if (!tiles.empty())
    BCU(b, cudaMemcpyAsync(b->base + b->tiles_off, tiles.data(), tiles.size() * sizeof(lbpc::BatchTile),
                           cudaMemcpyHostToDevice, b->stream),
        "batch work list upload");
  lbpc::BatchMeta m{(const lbpc::BatchTile*)(b->base + b->tiles_off), (int)tiles.size(), (int)b->inst.size()};
  BCU(b, cudaMemcpyAsync(b->base + b->meta_off, &m, sizeof m, cudaMemcpyHostToDevice, b->stream), "batch meta upload");
  for (int k = 0; k < (int)b->inst.size(); ++k) {
    lbpc_status s = upload_desc(b, k);
    if (s != LBPC_OK) return s;
  }
  BCU(b, cudaStreamSynchronize(b->stream), "batch rebuild sync");  // host staging of the copies is released
  b->dirty = false;
  ++b->gen;
  return LBPC_OK;
}

lbpc::SplitBuffers split_view(lbpc_batch* b, const HostInst& h, char* scratch) {
  lbpc::SplitBuffers s{};
  char* base = b->base + h.off;
  for (int j = 0; j < 2; ++j) {
    s.f[j] = base + h.f[j];
    s.g[j] = base + h.g[j];
    s.ref_f[j] = b->prec == LBPC_FP16DEV ? (float*)(base + h.rf[j]) : nullptr;
    s.ref_g[j] = b->prec == LBPC_FP16DEV ? (float*)(base + h.rg[j]) : nullptr;
    s.wall[j] = (double*)(base + h.wall[j]);
  }
  s.phi_prev = base + h.phi;
  s.partials = (double*)(base + h.partials);
  s.scalars = (double*)(base + h.scalars);
  s.status = (long long*)(b->base + b->status_off) + 8 * (&h - b->inst.data());
  if (scratch) {
    const size_t plane = a256((size_t)h.N * real_bytes(b->prec));
    for (int k = 0; k < lbpc::split_nplanes(); ++k) s.planes[k] = scratch + k * plane;
  }
  return s;
}

// One step as per-tile launches (ctas == 0): the active instances in launches of up to seg_capacity, each
// instance reading the buffer of parity h.cur ^ rel, then the per-instance advance. Whether the step is
// an instance's first comes from the host's count (h.step + rel), so lbpc_batch_step takes the first
// step of new instances outside the captured graphs.
template <class S> cudaError_t seg_step(lbpc_batch* b, int rel) {
  constexpr int CAP = lbpc::seg_capacity<S>(), SMALL = lbpc::kSegSmall;
  int tx, ty;
  lbpc::batch_tile_shape(b->variant, tx, ty);
  std::unique_ptr<lbpc::SegLaunch<S, CAP>> L(new lbpc::SegLaunch<S, CAP>());
  std::unique_ptr<lbpc::SegLaunch<S, SMALL>> Ls(new lbpc::SegLaunch<S, SMALL>());
  memset(L.get(), 0, sizeof(lbpc::SegLaunch<S, CAP>));
  int launches = 0;
  auto flush = [&]() -> cudaError_t {
    if (L->n == 0) return cudaSuccess;
    cudaError_t e;
    if (L->n <= SMALL) {  // the same records in the kernel with smaller parameters
      memset(Ls.get(), 0, sizeof(lbpc::SegLaunch<S, SMALL>));
      Ls->n = L->n;
      Ls->tiles = L->tiles;
      for (int j = 0; j < L->n; ++j) {
        Ls->first_tile[j] = L->first_tile[j];
        Ls->in[j] = L->in[j];
      }
      e = lbpc::batch_seg_launch(b->prec, b->variant, true, Ls.get(), launches > 0, b->stream);
    } else {
      e = lbpc::batch_seg_launch(b->prec, b->variant, false, L.get(), launches > 0, b->stream);
    }
    ++launches;
    L->n = 0;
    L->tiles = 0;
    return e;
  };
  for (int k = 0; k < (int)b->inst.size(); ++k) {
    const HostInst& h = b->inst[k];
    if (!h.used) continue;
    if (L->n == CAP) {
      const cudaError_t e = flush();
      if (e != cudaSuccess) return e;
    }
    L->first_tile[L->n] = L->tiles;
    lbpc::SegInst<S>& r = L->in[L->n++];
    char* base = b->base + h.off;
    const int c = h.cur ^ rel, d = c ^ 1;
    const bool half = b->prec == LBPC_FP16DEV;
    r.P = lbpc::params_of<typename lbpc::ArithOf<S>::type>(h.dp);
    r.fs = lbpc::PopBuf<S>{(S*)(base + h.f[c]), half ? (float*)(base + h.rf[c]) : nullptr, (double*)(base + h.wall[c])};
    r.gs = lbpc::PopBuf<S>{(S*)(base + h.g[c]), half ? (float*)(base + h.rg[c]) : nullptr, nullptr};
    r.fd = lbpc::PopBuf<S>{(S*)(base + h.f[d]), half ? (float*)(base + h.rf[d]) : nullptr, (double*)(base + h.wall[d])};
    r.gd = lbpc::PopBuf<S>{(S*)(base + h.g[d]), half ? (float*)(base + h.rg[d]) : nullptr, nullptr};
    r.phi_prev = base + h.phi;
    r.scalars = (double*)(base + h.scalars);
    r.partials = (double*)(base + h.partials);
    r.status = (long long*)(b->base + b->status_off) + 8 * k;
    r.step = (const long long*)(b->base + b->insts_off + (size_t)k * b->inst_struct + offsetof(lbpc::BatchInst<S>, step));
    r.tiles_x = (h.dp.nx + tx - 1) / tx;
    r.first = h.step + rel == 0;
    L->tiles += r.tiles_x * ((h.dp.ny + ty - 1) / ty);
  }
  const cudaError_t e = flush();
  if (e != cudaSuccess) return e;
  return lbpc::batch_advance_launch(b->prec, b->base + b->insts_off, (int)b->inst.size(), b->stream);
}

// One step of the current configuration; rel: parity of this step relative to the instances' h.cur.
cudaError_t launch_step(lbpc_batch* b, int rel) {
  if (b->ctas > 0)
    return lbpc::batch_step_launch(b->prec, b->variant, b->ctas, (const lbpc::BatchMeta*)(b->base + b->meta_off),
                                   b->base + b->insts_off, (int)b->inst.size(), b->stream);
  if (b->prec == LBPC_FP64) return seg_step<double>(b, rel);
  if (b->prec == LBPC_FP32) return seg_step<float>(b, rel);
  return seg_step<__half>(b, rel);
}

// The host's record of m steps taken by every instance.
void took_steps(lbpc_batch* b, int64_t m) {
  for (auto& h : b->inst)
    if (h.used) {
      h.step += m;
      h.cur ^= (int)(m & 1);
    }
  b->phase ^= (int)(m & 1);
}

// n steps launched one by one; rel0: parity of the first relative to the instances' h.cur.
lbpc_status launch_direct(lbpc_batch* b, int64_t n, int rel0) {
  for (int64_t k = 0; k < n; ++k) BCU(b, launch_step(b, (int)((rel0 + k) & 1)), "batch step launch");
  return LBPC_OK;
}

lbpc_status ensure_graph(lbpc_batch* b, cudaGraphExec_t* out) {
  const bool seg = b->ctas == 0;
  lbpc_batch::GraphSlot& s = b->graphs[seg ? b->phase : 0];
  if (s.exec && s.variant == b->variant && s.ctas == b->ctas && s.ninst == (int)b->inst.size() && (!seg || s.gen == b->gen)) {
    *out = s.exec;
    return LBPC_OK;
  }
  if (s.exec) {
    cudaGraphExecDestroy(s.exec);
    s.exec = nullptr;
  }
  cudaGraph_t g = nullptr;
  BCU(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "batch graph capture begin");
  cudaError_t le = cudaSuccess;
  for (int k = 0; k < b->chunk && le == cudaSuccess; ++k) le = launch_step(b, k & 1);
  const cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
  BCU(b, le, "batch graph capture launch");
  BCU(b, ce, "batch graph capture end");
  cudaError_t e = cudaGraphInstantiate(&s.exec, g, 0);
  cudaGraphDestroy(g);
  BCU(b, e, "batch graph instantiate");
  s.variant = b->variant;
  s.ctas = b->ctas;
  s.ninst = (int)b->inst.size();
  s.gen = b->gen;
  *out = s.exec;
  return LBPC_OK;
}

int active_count(const lbpc_batch* b) {
  int n = 0;
  for (auto& h : b->inst) n += h.used;
  return n;
}

}  // namespace

// ================================================================================================

LBPC_API size_t lbpc_batch_instance_bytes(const lbpc_params* p) {
  if (lbpc_check_params(p, nullptr, 0) != LBPC_OK) return 0;
  HostInst h;
  return a256(layout_instance(p, &h));
}

LBPC_API lbpc_status lbpc_batch_create(int32_t prec, int32_t max_instances, void* d_arena, size_t bytes, void* stream,
                                       lbpc_batch** out) {
  if (!out || !d_arena || max_instances <= 0 || max_instances > (1 << 20)) return LBPC_EINVAL;
  if (prec != LBPC_FP64 && prec != LBPC_FP32 && prec != LBPC_FP16DEV) return LBPC_EINVAL;
  if (((uintptr_t)d_arena & 255) != 0) return LBPC_EINVAL;
  *out = nullptr;
  lbpc_batch* b = new lbpc_batch();
  b->prec = prec;
  b->max_inst = max_instances;
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    delete b;
    return LBPC_ECUDA;
  }
  b->stream = (cudaStream_t)stream;
  b->base = (char*)d_arena;
  b->bytes = bytes;
  b->inst_struct = inst_struct_bytes(prec);
  b->arena.reset(bytes);
  const size_t fixed[3] = {sizeof(lbpc::BatchMeta), b->inst_struct * (size_t)max_instances,
                           8 * sizeof(long long) * (size_t)max_instances};
  size_t offs[3];
  for (int k = 0; k < 3; ++k)
    if (!b->arena.alloc(fixed[k], &offs[k])) {
      delete b;
      return LBPC_ENOMEM;
    }
  b->meta_off = offs[0];
  b->insts_off = offs[1];
  b->status_off = offs[2];
  {
    DevGuard g(b->device);
    if (cudaMemsetAsync(b->base + b->status_off, 0, fixed[2], b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->base + b->insts_off, 0, fixed[1], b->stream) != cudaSuccess) {
      delete b;
      return LBPC_ECUDA;
    }
    // default: per-tile launches of 32 x 8 tiles, the fastest configuration measured on uneven
    // instance mixes and on large instances in FP32, FP16 and FP64
    if (rebuild(b) != LBPC_OK) {
      delete b;
      return LBPC_ECUDA;
    }
  }
  *out = b;
  return LBPC_OK;
}

LBPC_API lbpc_status lbpc_batch_add(lbpc_batch* b, const lbpc_params* p, const double* rho, const double* T,
                                    int on_device, int32_t* id) {
  lbpc::TraceRange trace_("lbpc_batch_add");
  if (!b || !p || !rho || !T) return LBPC_EINVAL;
  if (b->err != LBPC_OK) return LBPC_ESTATE;
  char why[256];
  if (lbpc_check_params(p, why, sizeof why) != LBPC_OK) return bfail(b, LBPC_EINVAL, "lbpc_batch_add: %s", why);
  if (p->prec != b->prec) return bfail(b, LBPC_EINVAL, "lbpc_batch_add: prec %d differs from the batch's %d", p->prec, b->prec);
  if (9LL * p->nx * p->ny > 2147483647LL)  // the step kernel forms population indices in 32 bits
    return bfail(b, LBPC_EINVAL, "lbpc_batch_add: %d x %d nodes exceed a batch instance's 9 nx ny < 2^31", p->nx, p->ny);
  int slot = -1;
  for (int k = 0; k < (int)b->inst.size(); ++k)
    if (!b->inst[k].used) {
      slot = k;
      break;
    }
  if (slot < 0) {
    if ((int)b->inst.size() >= b->max_inst) return bfail(b, LBPC_ENOMEM, "lbpc_batch_add: all %d slots in use", b->max_inst);
    b->inst.emplace_back();
    slot = (int)b->inst.size() - 1;
  }
  HostInst h;
  h.p = *p;
  h.dp = lbpc::make_dev_params_public(p);
  h.N = (long long)p->nx * p->ny;
  h.bytes = layout_instance(p, &h);
  if (!b->arena.alloc(h.bytes, &h.off)) {
    if (slot == (int)b->inst.size() - 1 && !b->inst[slot].used) b->inst.pop_back();
    return bfail(b, LBPC_ENOMEM, "lbpc_batch_add: %zu bytes do not fit (largest free block %zu)", h.bytes, b->arena.largest());
  }
  h.used = true;
  b->inst[slot] = h;
  DevGuard g(b->device);
  HostInst& hi = b->inst[slot];
  lbpc::SplitBuffers s = split_view(b, hi, nullptr);
  const size_t nb = (size_t)hi.N * sizeof(double);
  const double *d_rho = rho, *d_T = T;
  if (!on_device) {  // stage in the B half; the init kernel writes the A half
    double* st = (double*)s.f[1];
    BCU(b, cudaMemcpyAsync(st, rho, nb, cudaMemcpyHostToDevice, b->stream), "lbpc_batch_add H2D rho");
    BCU(b, cudaMemcpyAsync(st + hi.N, T, nb, cudaMemcpyHostToDevice, b->stream), "lbpc_batch_add H2D T");
    d_rho = st;
    d_T = st + hi.N;
  }
  BCU(b, cudaMemsetAsync(s.status, 0, 8 * sizeof(long long), b->stream), "lbpc_batch_add status reset");
  BCU(b, lbpc::split_init(s, hi.dp, b->prec, d_rho, d_T, nullptr, nullptr, b->stream), "lbpc_batch_add init");
  hi.cur = 0;
  hi.step = 0;
  b->dirty = true;
  lbpc_status r = rebuild(b);
  if (r != LBPC_OK) return r;
  if (id) *id = slot;
  return LBPC_OK;
}

LBPC_API lbpc_status lbpc_batch_remove(lbpc_batch* b, int32_t id) {
  if (!b || id < 0 || id >= (int)b->inst.size() || !b->inst[id].used) return LBPC_EINVAL;
  DevGuard g(b->device);
  HostInst& h = b->inst[id];
  h.used = false;
  b->dirty = true;
  lbpc_status r = rebuild(b);  // synchronises: no launch reads the instance any more
  b->arena.release(h.off, h.bytes);
  return r;
}

LBPC_API lbpc_status lbpc_batch_step(lbpc_batch* b, int64_t n) {
  lbpc::TraceRange trace_("lbpc_batch_step");
  if (!b || n < 0) return LBPC_EINVAL;
  if (b->err != LBPC_OK) return LBPC_ESTATE;
  DevGuard g(b->device);
  if (b->dirty) {
    lbpc_status r = rebuild(b);
    if (r != LBPC_OK) return r;
  }
  int64_t left = n;
  if (left > 0 && b->ctas == 0) {  // per-tile launches take an instance's first step outside the graphs
    bool fresh = false;
    for (auto& h : b->inst) fresh |= h.used && h.step == 0;
    if (fresh) {
      lbpc_status r = launch_direct(b, 1, 0);
      if (r != LBPC_OK) return r;
      took_steps(b, 1);
      left -= 1;
    }
  }
  if (b->stream && left >= b->chunk) {
    cudaGraphExec_t exec = nullptr;
    lbpc_status r = ensure_graph(b, &exec);
    if (r != LBPC_OK) return r;
    while (left >= b->chunk) {
      BCU(b, cudaGraphLaunch(exec, b->stream), "batch graph launch");
      took_steps(b, b->chunk);
      left -= b->chunk;
    }
  }
  lbpc_status r = launch_direct(b, left, 0);
  if (r != LBPC_OK) return r;
  took_steps(b, left);
  return LBPC_OK;
}

LBPC_API lbpc_status lbpc_batch_check(lbpc_batch* b, int32_t* failed_id) {
  if (!b) return LBPC_EINVAL;
  if (failed_id) *failed_id = -1;
  DevGuard g(b->device);
  std::vector<long long> st(8 * b->inst.size());
  if (!st.empty())
    BCU(b, cudaMemcpyAsync(st.data(), b->base + b->status_off, st.size() * sizeof(long long), cudaMemcpyDeviceToHost,
                           b->stream),
        "batch status D2H");
  BCU(b, cudaStreamSynchronize(b->stream), "batch status sync");
  for (int k = 0; k < (int)b->inst.size(); ++k)
    if (b->inst[k].used && st[8 * k]) {
      if (failed_id) *failed_id = k;
      return bfail(b, LBPC_ENONPHYS, "instance %d: non-physical state at step %lld, node (x=%lld, y=%lld), code %lld", k,
                   st[8 * k + 1], st[8 * k + 2], st[8 * k + 3], st[8 * k + 4]);
    }
  return LBPC_OK;
}

LBPC_API lbpc_status lbpc_batch_fields(lbpc_batch* b, int32_t id, double* rho, double* ux, double* uy, double* T,
                                       int on_device) {
  lbpc::TraceRange trace_("lbpc_batch_fields");
  if (!b || id < 0 || id >= (int)b->inst.size() || !b->inst[id].used) return LBPC_EINVAL;
  DevGuard g(b->device);
  HostInst& h = b->inst[id];
  const size_t plane = a256((size_t)h.N * real_bytes(b->prec));
  const size_t sbytes = plane * lbpc::split_nplanes();
  size_t soff;
  if (!b->arena.alloc(sbytes, &soff)) return bfail(b, LBPC_ENOMEM, "lbpc_batch_fields: no room for %zu scratch bytes", sbytes);
  lbpc::SplitBuffers s = split_view(b, h, b->base + soff);
  const size_t nb = (size_t)h.N * sizeof(double);
  lbpc_status ret = LBPC_OK;
  if (on_device) {
    if (lbpc::split_fields(s, h.dp, b->prec, h.cur, h.step, rho, ux, uy, T, b->stream) != cudaSuccess) ret = LBPC_ECUDA;
  } else {
    double* st = (double*)s.f[h.cur ^ 1];  // dead half of the instance
    double* d[4] = {rho ? st : nullptr, ux ? st + h.N : nullptr, uy ? st + 2 * h.N : nullptr, T ? st + 3 * h.N : nullptr};
    if (lbpc::split_fields(s, h.dp, b->prec, h.cur, h.step, d[0], d[1], d[2], d[3], b->stream) != cudaSuccess)
      ret = LBPC_ECUDA;
    double* hh[4] = {rho, ux, uy, T};
    for (int k = 0; k < 4 && ret == LBPC_OK; ++k)
      if (hh[k] && cudaMemcpyAsync(hh[k], d[k], nb, cudaMemcpyDeviceToHost, b->stream) != cudaSuccess) ret = LBPC_ECUDA;
  }
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) ret = LBPC_ECUDA;
  b->arena.release(soff, sbytes);
  return ret == LBPC_OK ? LBPC_OK : bfail(b, ret, "lbpc_batch_fields failed");
}

LBPC_API lbpc_status lbpc_batch_sums(lbpc_batch* b, int32_t id, double* mass, double* heat) {
  if (!b || id < 0 || id >= (int)b->inst.size() || !b->inst[id].used) return LBPC_EINVAL;
  DevGuard g(b->device);
  HostInst& h = b->inst[id];
  lbpc::SplitBuffers s = split_view(b, h, nullptr);
  double v[2];
  BCU(b, lbpc::split_sums(s, h.dp, b->prec, h.cur, b->stream), "lbpc_batch_sums kernels");
  BCU(b, cudaMemcpyAsync(v, s.scalars + 1, sizeof v, cudaMemcpyDeviceToHost, b->stream), "lbpc_batch_sums D2H");
  BCU(b, cudaStreamSynchronize(b->stream), "lbpc_batch_sums sync");
  if (mass) *mass = v[0];
  if (heat) *heat = v[1];
  return LBPC_OK;
}

LBPC_API int64_t lbpc_batch_step_count(const lbpc_batch* b, int32_t id) {
  if (!b || id < 0 || id >= (int)b->inst.size() || !b->inst[id].used) return -1;
  return b->inst[id].step;
}

LBPC_API lbpc_status lbpc_batch_set_config(lbpc_batch* b, int32_t variant, int32_t ctas_per_sm) {
  if (!b || variant < 0 || variant >= lbpc::kBatchVariants || ctas_per_sm < 0) return LBPC_EINVAL;
  DevGuard g(b->device);
  const int occ = lbpc::batch_max_ctas_per_sm(b->prec, variant);
  if (occ < 1 || ctas_per_sm > 64 * occ)
    return bfail(b, LBPC_EINVAL, "ctas_per_sm %d above 64 times the residency limit %d", ctas_per_sm, occ);
  BCU(b, cudaStreamSynchronize(b->stream), "lbpc_batch_set_config sync");
  b->variant = variant;
  b->ctas = ctas_per_sm;
  b->dirty = true;
  return rebuild(b);
}

LBPC_API lbpc_status lbpc_batch_config(const lbpc_batch* b, int32_t* tile_x, int32_t* tile_y, int32_t* ctas_per_sm,
                                       int32_t* graph_chunk) {
  if (!b) return LBPC_EINVAL;
  int tx, ty;
  lbpc::batch_tile_shape(b->variant, tx, ty);
  if (tile_x) *tile_x = tx;
  if (tile_y) *tile_y = ty;
  if (ctas_per_sm) *ctas_per_sm = b->ctas;
  if (graph_chunk) *graph_chunk = b->chunk;
  return LBPC_OK;
}

LBPC_API lbpc_status lbpc_batch_autotune(lbpc_batch* b, int32_t steps_per_candidate, int32_t* best_variant,
                                         int32_t* best_ctas, float* best_ms_per_step) {
  lbpc::TraceRange trace_("lbpc_batch_autotune");
  if (!b || steps_per_candidate < 1) return LBPC_EINVAL;
  if (b->err != LBPC_OK) return LBPC_ESTATE;
  if (active_count(b) == 0) return bfail(b, LBPC_EINVAL, "lbpc_batch_autotune: the batch is empty");
  DevGuard g(b->device);
  cudaEvent_t e0, e1;
  BCU(b, cudaEventCreate(&e0), "autotune event");
  BCU(b, cudaEventCreate(&e1), "autotune event");
  float best = 1e30f;
  int bv = b->variant, bc = b->ctas;
  // whole graph chunks, so that every candidate is timed as lbpc_batch_step runs long step counts
  const int64_t timed = ((int64_t)std::max(steps_per_candidate, 1) + b->chunk - 1) / b->chunk * b->chunk;
  for (int v = 0; v < lbpc::kBatchVariants; ++v) {
    const int occ = lbpc::batch_max_ctas_per_sm(b->prec, v);
    // per-tile launches, the persistent grid, and grids of 16, 32 and 64 times it (the hardware then
    // balances tiles of uneven cost)
    std::vector<int> cand{0, occ, 16 * occ, 32 * occ, 64 * occ};
    for (int c : cand) {
      if (lbpc_batch_set_config(b, v, c) != LBPC_OK) continue;
      // every configuration computes the same step, so tuning advances the batch for real
      if (lbpc_batch_step(b, b->chunk) != LBPC_OK) break;  // warm-up: captures this candidate's graph
      BCU(b, cudaEventRecord(e0, b->stream), "autotune record");
      lbpc_status r = lbpc_batch_step(b, timed);
      BCU(b, cudaEventRecord(e1, b->stream), "autotune record");
      BCU(b, cudaEventSynchronize(e1), "autotune sync");
      if (r != LBPC_OK) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= (float)timed;
      if (ms < best) {
        best = ms;
        bv = v;
        bc = c;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  lbpc_status r = lbpc_batch_set_config(b, bv, bc);
  if (best_variant) *best_variant = bv;
  if (best_ctas) *best_ctas = bc;
  if (best_ms_per_step) *best_ms_per_step = best;
  return r;
}

LBPC_API int32_t lbpc_batch_per_tile_capacity(int32_t prec) {
  if (prec == LBPC_FP64) return lbpc::seg_capacity<double>();
  if (prec == LBPC_FP32) return lbpc::seg_capacity<float>();
  if (prec == LBPC_FP16DEV) return lbpc::seg_capacity<__half>();
  return 0;
}

LBPC_API size_t lbpc_batch_free_bytes(const lbpc_batch* b) { return b ? b->arena.free_bytes() : 0; }

LBPC_API const char* lbpc_batch_last_error(const lbpc_batch* b) { return b ? b->msg : "null batch"; }

LBPC_API void lbpc_batch_destroy(lbpc_batch* b) {
  if (!b) return;
  {
    DevGuard g(b->device);
    for (auto& s : b->graphs)
      if (s.exec) cudaGraphExecDestroy(s.exec);
  }
  delete b;
}
