"""Python binding of liblbpc (ctypes): argument marshalling only.

Every step of the computation runs in the CUDA kernels of liblbpc.so; this module fills the
``lbpc_params`` struct declared in ``include/lbpc.h``, allocates the caller-owned device workspace
with PyTorch, passes PyTorch's current CUDA stream, and moves FP64 fields in and out. There is no
CPU fallback: if the library is not built, or no CUDA device is present, the calls raise.
"""

import ctypes
import os
from dataclasses import dataclass, field
from typing import Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbpc.so")

LBPC_OK, LBPC_EINVAL, LBPC_ENOMEM, LBPC_ECUDA, LBPC_ENONPHYS, LBPC_ETIMEOUT, LBPC_ESTATE = range(7)
STATUS_NAMES = {0: "LBPC_OK", 1: "LBPC_EINVAL", 2: "LBPC_ENOMEM", 3: "LBPC_ECUDA", 4: "LBPC_ENONPHYS",
                5: "LBPC_ETIMEOUT", 6: "LBPC_ESTATE"}
FP64, FP32, FP16DEV, DF64 = 0, 1, 2, 3  # DF64: double-word (pairs of binary32) storage and arithmetic
PERIODIC, WALL, PRESSURE = 0, 1, 2
T_NONE, T_DIRICHLET = 0, 1
LAMBDA_CONST, LAMBDA_RHO_CV_CHI = 0, 1
IMPROVED, COMPROMISED, GONG_CHENG = 0, 1, 2
PATH_AUTO, PATH_SPLIT, PATH_FUSED = 0, 1, 2

EXPORTED = ["lbpc_version", "lbpc_check_params", "lbpc_workspace_bytes", "lbpc_eos_critical", "lbpc_coexistence",
            "lbpc_create", "lbpc_init", "lbpc_step", "lbpc_step_async", "lbpc_check", "lbpc_fields", "lbpc_sums",
            "lbpc_sums_async", "lbpc_populations", "lbpc_step_count", "lbpc_last_error", "lbpc_destroy", "lbpc_step_timed",
            "lbpc_kernel_name", "lbpc_set_path", "lbpc_step_static", "lbpc_batch_instance_bytes", "lbpc_batch_create",
            "lbpc_batch_add", "lbpc_batch_remove", "lbpc_batch_step", "lbpc_batch_check", "lbpc_batch_fields",
            "lbpc_batch_sums", "lbpc_batch_step_count", "lbpc_batch_set_config", "lbpc_batch_config",
            "lbpc_batch_autotune", "lbpc_batch_free_bytes", "lbpc_batch_last_error", "lbpc_batch_destroy",
            "lbpc_set_fused_tile", "lbpc_checkpoint_bytes", "lbpc_save", "lbpc_load", "lbpc_fma_rate",
            "lbpc_batch_per_tile_capacity"]


class LbpcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class CParams(ctypes.Structure):
    """Mirror of lbpc_params (include/lbpc.h); field order and types must match."""

    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("prec", ctypes.c_int32), ("model", ctypes.c_int32),
        ("lambda_mode", ctypes.c_int32), ("buoyancy", ctypes.c_int32),
        ("flow_bc", ctypes.c_int32 * 4), ("t_bc", ctypes.c_int32 * 4),
        ("strip_x0", ctypes.c_int32), ("strip_x1", ctypes.c_int32),
        ("a", ctypes.c_double), ("b", ctypes.c_double), ("R", ctypes.c_double), ("omega", ctypes.c_double),
        ("G", ctypes.c_double), ("s_f", ctypes.c_double * 9), ("s_g", ctypes.c_double * 9),
        ("sigma", ctypes.c_double), ("lambda_", ctypes.c_double), ("chi", ctypes.c_double), ("cV", ctypes.c_double),
        ("gx", ctypes.c_double), ("gy", ctypes.c_double), ("rho_bc", ctypes.c_double * 4),
        ("T_bc", ctypes.c_double * 4), ("T_strip", ctypes.c_double), ("G_wall", ctypes.c_double),
    ]


_lib_handle = None


def load_library(path: str = LIB_PATH):
    """Load liblbpc.so and declare its signatures. Raises if the library is missing."""
    global _lib_handle
    if _lib_handle is not None:
        return _lib_handle
    if not os.path.exists(path):
        raise RuntimeError(f"liblbpc.so is not built ({path}); run paper_1709_04400_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER(CParams)
    dp = ctypes.POINTER(ctypes.c_double)
    vp = ctypes.c_void_p
    sig = {
        "lbpc_version": (ctypes.c_int32, []),
        "lbpc_check_params": (ctypes.c_int, [P, ctypes.c_char_p, ctypes.c_size_t]),
        "lbpc_workspace_bytes": (ctypes.c_size_t, [P]),
        "lbpc_eos_critical": (ctypes.c_int, [P, dp, dp]),
        "lbpc_coexistence": (ctypes.c_int, [P, ctypes.c_double, dp, dp, dp]),
        "lbpc_create": (ctypes.c_int, [P, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]),
        "lbpc_init": (ctypes.c_int, [vp, vp, vp, vp, vp, ctypes.c_int]),
        "lbpc_step": (ctypes.c_int, [vp, ctypes.c_int64]),
        "lbpc_step_async": (ctypes.c_int, [vp, ctypes.c_int64]),
        "lbpc_check": (ctypes.c_int, [vp]),
        "lbpc_fields": (ctypes.c_int, [vp, vp, vp, vp, vp, ctypes.c_int]),
        "lbpc_sums": (ctypes.c_int, [vp, dp, dp]),
        "lbpc_sums_async": (ctypes.c_int, [vp, vp, ctypes.c_int]),
        "lbpc_populations": (ctypes.c_int, [vp, vp, vp, ctypes.c_int]),
        "lbpc_step_count": (ctypes.c_int64, [vp]),
        "lbpc_last_error": (ctypes.c_char_p, [vp]),
        "lbpc_destroy": (None, [vp]),
        "lbpc_step_timed": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_float), ctypes.c_int32,
                                           ctypes.POINTER(ctypes.c_int32)]),
        "lbpc_kernel_name": (ctypes.c_char_p, [vp, ctypes.c_int32]),
        "lbpc_set_path": (ctypes.c_int, [vp, ctypes.c_int32]),
        "lbpc_set_fused_tile": (ctypes.c_int, [vp, ctypes.c_int32]),
        "lbpc_checkpoint_bytes": (ctypes.c_size_t, [vp]),
        "lbpc_save": (ctypes.c_int, [vp, vp, ctypes.c_size_t, ctypes.c_int]),
        "lbpc_load": (ctypes.c_int, [vp, vp, ctypes.c_size_t, ctypes.c_int]),
        "lbpc_step_static": (ctypes.c_int, [P, vp, vp, vp, vp, vp, vp, vp, vp, ctypes.c_int64, vp]),
        "lbpc_fma_rate": (ctypes.c_int, [ctypes.c_int32, vp, dp]),
        "lbpc_batch_instance_bytes": (ctypes.c_size_t, [P]),
        "lbpc_batch_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]),
        "lbpc_batch_add": (ctypes.c_int, [vp, P, vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int32)]),
        "lbpc_batch_remove": (ctypes.c_int, [vp, ctypes.c_int32]),
        "lbpc_batch_step": (ctypes.c_int, [vp, ctypes.c_int64]),
        "lbpc_batch_check": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int32)]),
        "lbpc_batch_fields": (ctypes.c_int, [vp, ctypes.c_int32, vp, vp, vp, vp, ctypes.c_int]),
        "lbpc_batch_sums": (ctypes.c_int, [vp, ctypes.c_int32, dp, dp]),
        "lbpc_batch_step_count": (ctypes.c_int64, [vp, ctypes.c_int32]),
        "lbpc_batch_set_config": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.c_int32]),
        "lbpc_batch_config": (ctypes.c_int, [vp] + [ctypes.POINTER(ctypes.c_int32)] * 4),
        "lbpc_batch_autotune": (ctypes.c_int, [vp, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                               ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float)]),
        "lbpc_batch_per_tile_capacity": (ctypes.c_int32, [ctypes.c_int32]),
        "lbpc_batch_free_bytes": (ctypes.c_size_t, [vp]),
        "lbpc_batch_last_error": (ctypes.c_char_p, [vp]),
        "lbpc_batch_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib_handle = lib
    return lib


EDGE = {"x-": 0, "x+": 1, "y-": 2, "y+": 3}


@dataclass
class Params:
    """Physical and numerical parameters of a run (lattice units). Defaults are the paper's working
    point: Peng-Robinson a = 3/49, b = 2/21, R = 1, omega = 0.344 (after Eq. 56), nu = 0.1 and
    c_V = 5 (Sec. IV A), s_3 = s_5 = 1 (Sec. IV A)."""

    nx: int
    ny: int
    prec: int = FP64
    model: int = IMPROVED
    a: float = 3.0 / 49.0
    b: float = 2.0 / 21.0
    R: float = 1.0
    omega: float = 0.344
    G: float = -1.0
    s_f: Sequence[float] = (1.0, 0.8, 0.8, 1.0, 1.1, 1.0, 1.1, 1.25, 1.25)
    s_g: Sequence[float] = (1.0,) * 9
    sigma: float = 0.1
    lambda_mode: int = LAMBDA_CONST
    lam: float = 2.0 / 3.0
    chi: float = 0.06
    cV: float = 5.0
    gx: float = 0.0
    gy: float = 0.0
    buoyancy: int = 0  # 0 none, 1 (or True) F_b = (rho - rho_ave) g, 2 F_b = (rho - rho_bc[3]) g
    flow_bc: Sequence[int] = (PERIODIC,) * 4
    rho_bc: Sequence[float] = (0.0,) * 4
    t_bc: Sequence[int] = (T_NONE,) * 4
    T_bc: Sequence[float] = (0.0,) * 4
    strip: Optional[Tuple[int, int, float]] = None
    G_wall: float = 0.0

    @staticmethod
    def s_nu(nu):
        """Shear rate of the flow MRT: nu = c_s^2 (1/s_nu - 1/2)."""
        return 1.0 / (3.0 * nu + 0.5)

    def to_c(self) -> CParams:
        c = CParams()
        c.nx, c.ny, c.prec, c.model = self.nx, self.ny, self.prec, self.model
        c.lambda_mode, c.buoyancy = self.lambda_mode, int(self.buoyancy)  # True -> 1 (rho_ave), 2: top density
        c.flow_bc[:] = list(self.flow_bc)
        c.t_bc[:] = list(self.t_bc)
        if self.strip is not None:
            c.strip_x0, c.strip_x1, c.T_strip = int(self.strip[0]), int(self.strip[1]), float(self.strip[2])
        c.a, c.b, c.R, c.omega, c.G = self.a, self.b, self.R, self.omega, self.G
        c.s_f[:] = [float(v) for v in self.s_f]
        c.s_g[:] = [float(v) for v in self.s_g]
        c.sigma, c.lambda_, c.chi, c.cV = self.sigma, self.lam, self.chi, self.cV
        c.gx, c.gy, c.G_wall = self.gx, self.gy, self.G_wall
        c.rho_bc[:] = [float(v) for v in self.rho_bc]
        c.T_bc[:] = [float(v) for v in self.T_bc]
        return c


def check_params(p: Params):
    lib = load_library()
    buf = ctypes.create_string_buffer(256)
    c = p.to_c()
    s = lib.lbpc_check_params(ctypes.byref(c), buf, 256)
    return s, buf.value.decode()


def workspace_bytes(p: Params) -> int:
    c = p.to_c()
    return int(load_library().lbpc_workspace_bytes(ctypes.byref(c)))


def eos_critical(p: Params):
    c = p.to_c()
    Tc, pc = ctypes.c_double(), ctypes.c_double()
    s = load_library().lbpc_eos_critical(ctypes.byref(c), ctypes.byref(Tc), ctypes.byref(pc))
    if s != LBPC_OK:
        raise LbpcError(s, "lbpc_eos_critical")
    return Tc.value, pc.value


def fma_rate(prec=FP64, stream=None):
    """Measured FMA throughput of the current CUDA device in FLOP/s (lbpc_fma_rate): binary64 for FP64,
    binary32 for FP32. On PyTorch's current stream unless a torch.cuda.Stream is given."""
    import torch

    st = (stream or torch.cuda.current_stream()).cuda_stream
    out = ctypes.c_double()
    s = load_library().lbpc_fma_rate(int(prec), ctypes.c_void_p(st), ctypes.byref(out))
    if s != LBPC_OK:
        raise LbpcError(s, "lbpc_fma_rate")
    return out.value


def coexistence(p: Params, T: float):
    c = p.to_c()
    rv, rl, ps = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    s = load_library().lbpc_coexistence(ctypes.byref(c), float(T), ctypes.byref(rv), ctypes.byref(rl), ctypes.byref(ps))
    if s != LBPC_OK:
        raise LbpcError(s, f"lbpc_coexistence(T={T})")
    return rv.value, rl.value, ps.value


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data) if isinstance(a, np.ndarray) else ctypes.c_void_p(a.data_ptr())


class Simulation:
    """One simulation on one CUDA device: a context of liblbpc over a PyTorch-owned workspace."""

    def __init__(self, params: Params, device=None, stream=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("liblbpc needs a CUDA device; none is available")
        self.lib = load_library()
        self.params = params
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self._c = params.to_c()
        nbytes = int(self.lib.lbpc_workspace_bytes(ctypes.byref(self._c)))
        if nbytes == 0:
            s, msg = check_params(params)
            raise LbpcError(s, msg)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.stream = torch.cuda.current_stream(self.device) if stream is None else stream
            ctx = ctypes.c_void_p()
            s = self.lib.lbpc_create(ctypes.byref(self._c), ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                     ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx))
        if s != LBPC_OK:
            raise LbpcError(s, "lbpc_create")
        self.ctx = ctx
        self.nx, self.ny = params.nx, params.ny

    # -- helpers ------------------------------------------------------------------------------
    def _raise(self, s, what):
        if s != LBPC_OK:
            raise LbpcError(s, f"{what}: {self.lib.lbpc_last_error(self.ctx).decode()}")

    def _host(self, a):
        if a is None:
            return None
        a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(self.ny, self.nx))
        return a

    # -- API ----------------------------------------------------------------------------------
    def init(self, rho, T, ux=None, uy=None):
        """Equilibrium start from FP64 fields: numpy arrays (host) or CUDA tensors (device)."""
        import torch

        if isinstance(rho, torch.Tensor):
            for name, x in zip(("rho", "T", "ux", "uy"), (rho, T, ux, uy)):
                if x is not None and x.numel() != self.nx * self.ny:  # the kernels read nx * ny values
                    raise ValueError(f"{name} has {x.numel()} values, the grid {self.ny} x {self.nx}")
            args = [x if x is None else x.to(device=self.device, dtype=torch.float64).contiguous() for x in (rho, T, ux, uy)]
            ptrs = [ctypes.c_void_p(0) if x is None else ctypes.c_void_p(x.data_ptr()) for x in args]
            self._keep = args
            s = self.lib.lbpc_init(self.ctx, *ptrs, 1)
        else:
            args = [self._host(x) for x in (rho, T, ux, uy)]
            ptrs = [ctypes.c_void_p(0) if x is None else _ptr(x) for x in args]
            s = self.lib.lbpc_init(self.ctx, *ptrs, 0)
        self._raise(s, "lbpc_init")

    def set_path(self, path):
        """Kernel organisation of the step: PATH_AUTO, PATH_SPLIT or PATH_FUSED."""
        self._raise(self.lib.lbpc_set_path(self.ctx, int(path)), "lbpc_set_path")

    def set_fused_tile(self, tile):
        """Tile configuration of the fused step (lbpc_set_fused_tile): 0 = 32 x 16, 1 = 32 x 8, 2 / 3 = 32 x 16 /
        32 x 32 with two nodes per thread, 4 = 32 x 8 in persistent CTAs staging ahead (default)."""
        self._raise(self.lib.lbpc_set_fused_tile(self.ctx, int(tile)), "lbpc_set_fused_tile")

    def step(self, n=1, sync=True):
        s = (self.lib.lbpc_step if sync else self.lib.lbpc_step_async)(self.ctx, int(n))
        self._raise(s, "lbpc_step")

    def step_timed(self):
        """One step; returns {kernel name: launch duration in ms} measured with CUDA events on the
        context's stream."""
        ms = (ctypes.c_float * 16)()
        n = ctypes.c_int32()
        self._raise(self.lib.lbpc_step_timed(self.ctx, ms, 16, ctypes.byref(n)), "lbpc_step_timed")
        return {self.lib.lbpc_kernel_name(self.ctx, k).decode(): float(ms[k]) for k in range(n.value)}

    def check(self):
        self._raise(self.lib.lbpc_check(self.ctx), "lbpc_check")

    def fields(self, device=False):
        """(rho, ux, uy, T) of the current state as [ny][nx] FP64 numpy arrays (or CUDA tensors)."""
        import torch

        if device:
            out = [torch.empty((self.ny, self.nx), dtype=torch.float64, device=self.device) for _ in range(4)]
            s = self.lib.lbpc_fields(self.ctx, *[ctypes.c_void_p(t.data_ptr()) for t in out], 1)
        else:
            out = [np.empty((self.ny, self.nx)) for _ in range(4)]
            s = self.lib.lbpc_fields(self.ctx, *[_ptr(a) for a in out], 0)
        self._raise(s, "lbpc_fields")
        return tuple(out)

    def sums_async(self, out):
        """Enqueue the domain sums and a copy of (mass, heat) into out, a 2-element float64 CUDA tensor
        or pinned host tensor, without waiting (lbpc_sums_async)."""
        import torch

        if out.dtype != torch.float64 or out.numel() < 2 or not out.is_contiguous():
            raise ValueError("sums_async needs a contiguous float64 tensor of at least 2 elements")
        self._raise(self.lib.lbpc_sums_async(self.ctx, ctypes.c_void_p(out.data_ptr()), int(out.is_cuda)),
                    "lbpc_sums_async")

    def sums(self):
        m, h = ctypes.c_double(), ctypes.c_double()
        self._raise(self.lib.lbpc_sums(self.ctx, ctypes.byref(m), ctypes.byref(h)), "lbpc_sums")
        return m.value, h.value

    def save(self, out=None):
        """Checkpoint of the whole state (lbpc_save) into a host numpy uint8 array or, when out is a
        CUDA uint8 tensor of at least checkpoint_bytes(), into it; returns the buffer."""
        n = self.lib.lbpc_checkpoint_bytes(self.ctx)
        if out is None:
            out = np.empty(n, dtype=np.uint8)
        dev = not isinstance(out, np.ndarray)
        self._raise(self.lib.lbpc_save(self.ctx, _ptr(out), int(out.numel() if dev else out.size), int(dev)),
                    "lbpc_save")
        return out

    def load(self, buf):
        """Restore a checkpoint (lbpc_load) from a host numpy uint8 array or a CUDA uint8 tensor."""
        dev = not isinstance(buf, np.ndarray)
        if not dev:
            buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._raise(self.lib.lbpc_load(self.ctx, _ptr(buf), int(buf.numel() if dev else buf.size), int(dev)),
                    "lbpc_load")

    def checkpoint_bytes(self):
        return int(self.lib.lbpc_checkpoint_bytes(self.ctx))

    def populations(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((9, self.ny, self.nx))
        self._raise(self.lib.lbpc_populations(self.ctx, _ptr(f), _ptr(g), 0), "lbpc_populations")
        return f, g

    @property
    def step_count(self):
        return int(self.lib.lbpc_step_count(self.ctx))

    def last_error(self):
        return self.lib.lbpc_last_error(self.ctx).decode()

    def close(self):
        if getattr(self, "ctx", None) is not None:
            self.lib.lbpc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_FLOW = {"periodic": PERIODIC, "wall": WALL, "pressure": PRESSURE}
_TBC = {"none": T_NONE, "dirichlet": T_DIRICHLET}
_LAM = {"const": LAMBDA_CONST, "rho_cv_chi": LAMBDA_RHO_CV_CHI}
_MODEL = {"improved": IMPROVED, "compromised": COMPROMISED, "gong_cheng": GONG_CHENG}


def params_from_case(case: dict, prec: int = FP64) -> Params:
    """Params from a workload dict (see paper_1709_04400_gb300.workloads)."""
    return Params(
        nx=case["nx"], ny=case["ny"], prec=prec, model=_MODEL[case.get("model", "improved")],
        s_f=case["s_f"], s_g=case["s_g"], sigma=case["sigma"], lambda_mode=_LAM[case["lambda_mode"]],
        lam=case.get("lam", 0.0), chi=case.get("chi", 0.06), cV=case["cV"], gx=case.get("gx", 0.0),
        gy=case.get("gy", 0.0), buoyancy=case.get("buoyancy", False),
        flow_bc=[_FLOW[k] for k in case["flow_bc"]], rho_bc=case.get("rho_bc", (0.0,) * 4),
        t_bc=[_TBC[k] for k in case["t_bc"]], T_bc=case.get("T_bc", (0.0,) * 4), strip=case.get("strip"),
        G_wall=case.get("G_wall", 0.0))


class Batch:
    """Many simulations advancing together (lbpc_batch_*): per-tile launches that hold the instances in
    their parameters, or one work-list launch per step (set_config), replayed through CUDA graphs on a
    dedicated stream. The arena is a PyTorch uint8 buffer of arena_bytes."""

    def __init__(self, prec: int, arena_bytes: int, max_instances: int = 4096, device=None, high_priority=False):
        """high_priority: the batch's stream takes the device's highest stream priority, so that its CTAs are
        dispatched first when other work shares the GPU (a serving batch beside bulk simulations)."""
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("liblbpc needs a CUDA device; none is available")
        self.lib = load_library()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.prec = prec
        with torch.cuda.device(self.device):
            self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=self.device)
            prio = torch.cuda.Stream.priority_range()[1] if high_priority else 0
            self.stream = torch.cuda.Stream(self.device, priority=prio)
        h = ctypes.c_void_p()
        s = self.lib.lbpc_batch_create(prec, max_instances, ctypes.c_void_p(self.arena.data_ptr()), int(arena_bytes),
                                       ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        if s != LBPC_OK:
            raise LbpcError(s, "lbpc_batch_create")
        self.h = h
        self.shapes = {}

    def _raise(self, s, what):
        if s != LBPC_OK:
            raise LbpcError(s, f"{what}: {self.lib.lbpc_batch_last_error(self.h).decode()}")

    @staticmethod
    def per_tile_capacity(prec: int) -> int:
        """Instances one per-tile launch (configuration with 0 CTAs per SM) holds."""
        return int(load_library().lbpc_batch_per_tile_capacity(int(prec)))

    @staticmethod
    def instance_bytes(params: Params) -> int:
        c = params.to_c()
        return int(load_library().lbpc_batch_instance_bytes(ctypes.byref(c)))

    def add(self, params: Params, rho, T) -> int:
        c = params.to_c()
        rho = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).reshape(params.ny, params.nx))
        T = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(params.ny, params.nx))
        i = ctypes.c_int32()
        self._raise(self.lib.lbpc_batch_add(self.h, ctypes.byref(c), _ptr(rho), _ptr(T), 0, ctypes.byref(i)),
                    "lbpc_batch_add")
        self.shapes[i.value] = (params.ny, params.nx)
        return i.value

    def remove(self, i: int):
        self._raise(self.lib.lbpc_batch_remove(self.h, int(i)), "lbpc_batch_remove")
        self.shapes.pop(i, None)

    def step(self, n: int = 1):
        self._raise(self.lib.lbpc_batch_step(self.h, int(n)), "lbpc_batch_step")

    def check(self):
        f = ctypes.c_int32()
        s = self.lib.lbpc_batch_check(self.h, ctypes.byref(f))
        if s != LBPC_OK:
            err = LbpcError(s, self.lib.lbpc_batch_last_error(self.h).decode())
            err.instance = f.value
            raise err

    def fields(self, i: int):
        ny, nx = self.shapes[i]
        out = [np.empty((ny, nx)) for _ in range(4)]
        self._raise(self.lib.lbpc_batch_fields(self.h, int(i), *[_ptr(a) for a in out], 0), "lbpc_batch_fields")
        return tuple(out)

    def sums(self, i: int):
        m, h = ctypes.c_double(), ctypes.c_double()
        self._raise(self.lib.lbpc_batch_sums(self.h, int(i), ctypes.byref(m), ctypes.byref(h)), "lbpc_batch_sums")
        return m.value, h.value

    def step_count(self, i: int) -> int:
        return int(self.lib.lbpc_batch_step_count(self.h, int(i)))

    def set_config(self, variant: int, ctas_per_sm: int):
        self._raise(self.lib.lbpc_batch_set_config(self.h, int(variant), int(ctas_per_sm)), "lbpc_batch_set_config")

    def config(self):
        v = [ctypes.c_int32() for _ in range(4)]
        self._raise(self.lib.lbpc_batch_config(self.h, *[ctypes.byref(x) for x in v]), "lbpc_batch_config")
        return dict(tile_x=v[0].value, tile_y=v[1].value, ctas_per_sm=v[2].value, graph_chunk=v[3].value)

    def autotune(self, steps_per_candidate: int = 4):
        bv, bc, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
        self._raise(self.lib.lbpc_batch_autotune(self.h, int(steps_per_candidate), ctypes.byref(bv), ctypes.byref(bc),
                                                 ctypes.byref(ms)), "lbpc_batch_autotune")
        return dict(variant=bv.value, ctas_per_sm=bc.value, ms_per_step=ms.value)

    def free_bytes(self) -> int:
        return int(self.lib.lbpc_batch_free_bytes(self.h))

    def synchronize(self):
        self.stream.synchronize()

    def close(self):
        if getattr(self, "h", None) is not None:
            self.stream.synchronize()
            self.lib.lbpc_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
