"""Thin ctypes binding of libgbfd (include/gbfd.h): same names, argument
marshalling only.  Every step of the solver runs in the library's CUDA
kernels; there is no CPU path.  PyTorch provides the device workspace and
the stream.

Low-level functions mirror the C ABI one to one (``gbfd_init``,
``gbfd_rk3_step``, ...) and raise ``GbfdError`` on a non-OK status.
``Solver`` bundles a context with its torch-allocated workspace.
"""
import ctypes
import os

import numpy as np

from . import build as _build

GBFD_OK = 0
STATUS = {0: "GBFD_OK", 1: "GBFD_ERR_INVALID_ARG", 2: "GBFD_ERR_WORKSPACE", 3: "GBFD_ERR_CUDA",
          4: "GBFD_ERR_TIMEOUT", 5: "GBFD_ERR_UNSUPPORTED", 6: "GBFD_ERR_STATE"}

GBFD_FP64, GBFD_FP32, GBFD_FP32_ACC64, GBFD_FP32_ACC64_W64, GBFD_FP32_ACCFF = 0, 1, 2, 3, 4
GBFD_55P, GBFD_19P = 0, 1
GBFD_OPT_KERNEL_PATH, GBFD_OPT_TILE_CONFIG, GBFD_OPT_FAULT_SKIP_COPY, GBFD_OPT_HOST_PATH = 1, 2, 3, 4
GBFD_OPT_HOST_ASYNC = 5
GBFD_BC_PERIODIC, GBFD_BC_WALL, GBFD_BC_EXCHANGE = 0, 1, 2
BCS = {"periodic": GBFD_BC_PERIODIC, "wall": GBFD_BC_WALL, "exchange": GBFD_BC_EXCHANGE}

PRECISIONS = {"fp64": GBFD_FP64, "fp32": GBFD_FP32, "fp32_acc64": GBFD_FP32_ACC64,
              "fp32_acc64_w64": GBFD_FP32_ACC64_W64, "fp32_accff": GBFD_FP32_ACCFF}
FORMS = {"55p": GBFD_55P, "19p": GBFD_19P}

# exported symbols of include/gbfd.h (checked by the ABI test)
EXPORTS = ("gbfd_workspace_bytes", "gbfd_init", "gbfd_destroy", "gbfd_set_state",
           "gbfd_get_state", "gbfd_rk3_step", "gbfd_rk3_step_forced", "gbfd_substep", "gbfd_diagnostics", "gbfd_cfl_dt",
           "gbfd_sync", "gbfd_set_option", "gbfd_launch_count", "gbfd_last_error",
           "gbfd_status_string", "gbfd_diagnostics_noalloc", "gbfd_autotune",
           "gbfd_batch_workspace_bytes", "gbfd_batch_init", "gbfd_batch_destroy",
           "gbfd_batch_set_state", "gbfd_batch_get_state", "gbfd_batch_step",
           "gbfd_batch_diagnostics", "gbfd_batch_sync", "gbfd_batch_set_option",
           "gbfd_batch_autotune", "gbfd_batch_launch_count", "gbfd_batch_last_error",
           "gbfd_cnn_workspace_bytes", "gbfd_cnn_init", "gbfd_cnn_destroy",
           "gbfd_cnn_param_count", "gbfd_cnn_set_params", "gbfd_cnn_get_params",
           "gbfd_cnn_set_norm", "gbfd_cnn_forward", "gbfd_cnn_gradients",
           "gbfd_cnn_train_step", "gbfd_cnn_apply", "gbfd_step_corrected", "gbfd_box_filter",
           "gbfd_cnn_launch_count", "gbfd_cnn_last_error", "gbfd_cnn_set_option",
           "gbfd_fp64_fma_rate", "gbfd_tc_mma_cycles", "gbfd_halo_bytes", "gbfd_halo_pack", "gbfd_halo_unpack",
           "gbfd_batch_get_option")
GBFD_CNN_OPT_CONV_GRID, GBFD_CNN_OPT_WGRAD_PARTS = 1, 2
GBFD_BATCH_OPT_GRAPH, GBFD_BATCH_OPT_ZCHUNK, GBFD_BATCH_OPT_GRID = 1, 2, 3
GBFD_BATCH_OPT_KERNEL, GBFD_BATCH_OPT_DATAFLOW, GBFD_BATCH_OPT_FAULT_STALL = 4, 5, 6


class GbfdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class gbfd_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("form", ctypes.c_int32),
                ("entropy_mode", ctypes.c_int32), ("lx", ctypes.c_double),
                ("ly", ctypes.c_double), ("lz", ctypes.c_double), ("cs", ctypes.c_double),
                ("nu", ctypes.c_double), ("bc_z", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class gbfd_diag(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("ekin", ctypes.c_double),
                ("umax", ctypes.c_double), ("urms", ctypes.c_double),
                ("rms", ctypes.c_double * 5), ("maxabs", ctypes.c_double * 5),
                ("nonfinite", ctypes.c_int32), ("nfields", ctypes.c_int32)]

    def as_dict(self):
        return {"mass": self.mass, "ekin": self.ekin, "umax": self.umax, "urms": self.urms,
                "rms": np.array(self.rms[:]), "maxabs": np.array(self.maxabs[:]),
                "nonfinite": int(self.nonfinite), "nfields": int(self.nfields)}


_lib = None
_VP = ctypes.c_void_p


def library_path():
    return _build.LIB


def load(path=None):
    """Open libgbfd.so (built by ``build.build()``); raises OSError if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise OSError(f"libgbfd.so not built ({path}); run __graft_entry__.build()")
    L = ctypes.CDLL(path)
    L.gbfd_workspace_bytes.restype = ctypes.c_size_t
    L.gbfd_workspace_bytes.argtypes = [ctypes.POINTER(gbfd_params)]
    L.gbfd_init.argtypes = [ctypes.POINTER(gbfd_params), _VP, ctypes.c_size_t, _VP,
                            ctypes.POINTER(_VP)]
    L.gbfd_destroy.argtypes = [_VP]
    L.gbfd_set_state.argtypes = [_VP, _VP, ctypes.c_int, ctypes.c_int]
    L.gbfd_get_state.argtypes = [_VP, _VP, ctypes.c_int, ctypes.c_int]
    L.gbfd_rk3_step.argtypes = [_VP, ctypes.c_double, ctypes.c_int]
    L.gbfd_rk3_step_forced.argtypes = [_VP, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_double),
                                       ctypes.POINTER(ctypes.c_double)]
    L.gbfd_substep.argtypes = [_VP, ctypes.c_int, ctypes.c_double]
    L.gbfd_diagnostics.argtypes = [_VP, ctypes.POINTER(gbfd_diag)]
    L.gbfd_cfl_dt.argtypes = [_VP, ctypes.c_double, ctypes.c_double,
                              ctypes.POINTER(ctypes.c_double)]
    L.gbfd_sync.argtypes = [_VP]
    L.gbfd_set_option.argtypes = [_VP, ctypes.c_int, ctypes.c_int64]
    L.gbfd_launch_count.restype = ctypes.c_int64
    L.gbfd_launch_count.argtypes = [_VP]
    L.gbfd_last_error.restype = ctypes.c_char_p
    L.gbfd_last_error.argtypes = [_VP]
    L.gbfd_diagnostics_noalloc.argtypes = [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, _VP, _VP]
    L.gbfd_autotune.argtypes = [_VP, ctypes.c_int, ctypes.c_char_p, ctypes.POINTER(ctypes.c_int),
                                ctypes.POINTER(ctypes.c_double)]
    _I32P = ctypes.POINTER(ctypes.c_int32)
    _DP = ctypes.POINTER(ctypes.c_double)
    L.gbfd_batch_workspace_bytes.restype = ctypes.c_size_t
    L.gbfd_batch_workspace_bytes.argtypes = [ctypes.c_int, _I32P, ctypes.c_int]
    L.gbfd_batch_init.argtypes = [ctypes.c_int, _I32P, _DP, _DP, ctypes.c_double, ctypes.c_int,
                                  _VP, ctypes.c_size_t, _VP, ctypes.POINTER(_VP)]
    L.gbfd_batch_destroy.argtypes = [_VP]
    L.gbfd_batch_set_state.argtypes = [_VP, ctypes.c_int, _VP, ctypes.c_int, ctypes.c_int]
    L.gbfd_batch_get_state.argtypes = [_VP, ctypes.c_int, _VP, ctypes.c_int, ctypes.c_int]
    L.gbfd_batch_step.argtypes = [_VP, _DP, ctypes.c_int]
    L.gbfd_batch_diagnostics.argtypes = [_VP, ctypes.c_int, ctypes.POINTER(gbfd_diag)]
    L.gbfd_batch_sync.argtypes = [_VP]
    L.gbfd_batch_set_option.argtypes = [_VP, ctypes.c_int, ctypes.c_int64]
    L.gbfd_batch_get_option.argtypes = [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]
    L.gbfd_batch_autotune.argtypes = [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_int), _DP]
    L.gbfd_batch_launch_count.restype = ctypes.c_int64
    L.gbfd_batch_launch_count.argtypes = [_VP]
    L.gbfd_batch_last_error.restype = ctypes.c_char_p
    L.gbfd_batch_last_error.argtypes = [_VP]
    _FP = ctypes.POINTER(ctypes.c_float)
    L.gbfd_cnn_workspace_bytes.restype = ctypes.c_size_t
    L.gbfd_cnn_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int]
    L.gbfd_cnn_init.argtypes = [ctypes.c_int, ctypes.c_int, _VP, ctypes.c_size_t, _VP,
                                ctypes.POINTER(_VP)]
    L.gbfd_cnn_destroy.argtypes = [_VP]
    L.gbfd_cnn_param_count.argtypes = []
    L.gbfd_cnn_set_params.argtypes = [_VP, _FP]
    L.gbfd_cnn_get_params.argtypes = [_VP, _FP]
    L.gbfd_cnn_set_norm.argtypes = [_VP, _FP, _FP, _FP]
    L.gbfd_cnn_forward.argtypes = [_VP, _VP, ctypes.c_int, ctypes.c_int, _VP]
    L.gbfd_cnn_gradients.argtypes = [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, _FP, _DP]
    L.gbfd_cnn_train_step.argtypes = [_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                      _DP]
    L.gbfd_cnn_apply.argtypes = [_VP, _VP]
    L.gbfd_step_corrected.argtypes = [_VP, _VP, ctypes.c_double, ctypes.c_int]
    L.gbfd_box_filter.argtypes = [_VP, ctypes.c_int, _VP]
    L.gbfd_cnn_launch_count.restype = ctypes.c_int64
    L.gbfd_cnn_launch_count.argtypes = [_VP]
    L.gbfd_cnn_last_error.restype = ctypes.c_char_p
    L.gbfd_cnn_last_error.argtypes = [_VP]
    L.gbfd_cnn_set_option.argtypes = [_VP, ctypes.c_int, ctypes.c_int64]
    L.gbfd_fp64_fma_rate.argtypes = [_VP, _DP]
    L.gbfd_tc_mma_cycles.argtypes = [ctypes.c_int, _VP, _DP]
    L.gbfd_halo_bytes.restype = ctypes.c_size_t
    L.gbfd_halo_bytes.argtypes = [_VP]
    L.gbfd_halo_pack.argtypes = [_VP, ctypes.c_int, _VP]
    L.gbfd_halo_unpack.argtypes = [_VP, ctypes.c_int, _VP]
    L.gbfd_status_string.restype = ctypes.c_char_p
    L.gbfd_status_string.argtypes = [ctypes.c_int]
    for name in EXPORTS:
        getattr(L, name).restype = getattr(L, name).restype or ctypes.c_int
    _lib = L
    return L


def _check(status, ctx=None):
    if status != GBFD_OK:
        msg = load().gbfd_last_error(ctx).decode(errors="replace")
        raise GbfdError(status, msg)


# ------------------------------------------------------------ C-ABI mirror

def gbfd_workspace_bytes(params):
    return load().gbfd_workspace_bytes(ctypes.byref(params))


def gbfd_init(params, workspace_ptr, workspace_bytes, stream_ptr):
    ctx = _VP()
    _check(load().gbfd_init(ctypes.byref(params), _VP(workspace_ptr), workspace_bytes,
                            _VP(stream_ptr), ctypes.byref(ctx)))
    return ctx


def gbfd_destroy(ctx):
    _check(load().gbfd_destroy(ctx))


def gbfd_set_state(ctx, src_ptr, src_on_device, src_is_fp64):
    _check(load().gbfd_set_state(ctx, _VP(src_ptr), int(src_on_device), int(src_is_fp64)), ctx)


def gbfd_get_state(ctx, dst_ptr, dst_on_device, dst_is_fp64):
    _check(load().gbfd_get_state(ctx, _VP(dst_ptr), int(dst_on_device), int(dst_is_fp64)), ctx)


def gbfd_rk3_step(ctx, dt, nsteps):
    _check(load().gbfd_rk3_step(ctx, float(dt), int(nsteps)), ctx)


def gbfd_rk3_step_forced(ctx, dt, f0, k, phi, e):
    """len(phi) forced RK3 steps: k (n, 3) integers, phi (n,), e (n, 3)."""
    k = np.ascontiguousarray(np.asarray(k).reshape(-1, 3), dtype=np.int32)
    phi = np.ascontiguousarray(np.asarray(phi, dtype=np.float64).reshape(-1))
    e = np.ascontiguousarray(np.asarray(e, dtype=np.float64).reshape(-1, 3))
    n = phi.shape[0]
    assert k.shape[0] == n and e.shape[0] == n
    _check(load().gbfd_rk3_step_forced(
        ctx, float(dt), int(n), float(f0), k.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
        phi.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), ctx)


def gbfd_substep(ctx, s, dt):
    _check(load().gbfd_substep(ctx, int(s), float(dt)), ctx)


def gbfd_diagnostics(ctx):
    d = gbfd_diag()
    _check(load().gbfd_diagnostics(ctx, ctypes.byref(d)), ctx)
    return d


def gbfd_cfl_dt(ctx, cfl=0.4, cnu=0.25):
    out = ctypes.c_double()
    _check(load().gbfd_cfl_dt(ctx, cfl, cnu, ctypes.byref(out)), ctx)
    return out.value


def gbfd_sync(ctx):
    _check(load().gbfd_sync(ctx), ctx)


def gbfd_set_option(ctx, key, value):
    _check(load().gbfd_set_option(ctx, int(key), int(value)), ctx)


def gbfd_launch_count(ctx):
    return load().gbfd_launch_count(ctx)


def gbfd_diagnostics_noalloc(state_ptr, state_is_fp64, nx, ny, nz, nfields, lx, ly, lz,
                             stream_ptr, out_ptr):
    """Diagnostics of a device state array into a device buffer of 16 doubles,
    without a context, a workspace or any allocation (see include/gbfd.h)."""
    _check(load().gbfd_diagnostics_noalloc(_VP(state_ptr), int(state_is_fp64), nx, ny, nz,
                                           nfields, lx, ly, lz, _VP(stream_ptr), _VP(out_ptr)))


def gbfd_autotune(ctx, reps=3, cache_path=None):
    """Pick the fastest tile configuration (see include/gbfd.h); returns
    (table index, ms per RK3 step, 0.0 on a cache hit)."""
    cfg = ctypes.c_int()
    ms = ctypes.c_double()
    path = cache_path.encode() if cache_path else None
    _check(load().gbfd_autotune(ctx, int(reps), path, ctypes.byref(cfg), ctypes.byref(ms)), ctx)
    return cfg.value, ms.value


def gbfd_fp64_fma_rate(stream_ptr=None):
    """Measured FP64 FMA rate of the current device in TFLOP/s (the FP64
    path's roofline denominator)."""
    if stream_ptr is None:
        import torch
        stream_ptr = torch.cuda.current_stream().cuda_stream
    r = ctypes.c_double()
    _check(load().gbfd_fp64_fma_rate(_VP(stream_ptr), ctypes.byref(r)))
    return r.value


def gbfd_tc_mma_cycles(n, stream_ptr=None):
    """SM clock cycles per tcgen05 MMA of M = 128, K = 16 and N = n columns
    (BF16 from shared memory), measured on the current device."""
    if stream_ptr is None:
        import torch
        stream_ptr = torch.cuda.current_stream().cuda_stream
    r = ctypes.c_double()
    _check(load().gbfd_tc_mma_cycles(int(n), _VP(stream_ptr), ctypes.byref(r)))
    return r.value


def gbfd_last_error(ctx=None):
    return load().gbfd_last_error(ctx).decode(errors="replace")


# ------------------------------------------------------------ convenience

def make_params(shape, lengths=(2 * np.pi,) * 3, cs=1.0, nu=5e-3, precision="fp64", form="55p",
                entropy_mode=1, bc_z="periodic"):
    nz, ny, nx = shape
    p = gbfd_params()
    p.bc_z = BCS[bc_z] if isinstance(bc_z, str) else int(bc_z)
    p.nx, p.ny, p.nz = nx, ny, nz
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.form = FORMS[form] if isinstance(form, str) else int(form)
    p.entropy_mode = int(entropy_mode)
    p.lx, p.ly, p.lz = lengths
    p.cs, p.nu = cs, nu
    return p


class Solver:
    """A gbfd context plus its workspace (a torch CUDA uint8 tensor).

    State arrays are (nfields, nz, ny, nx); nfields = 5 with entropy_mode 1,
    4 with entropy_mode 0.  bc_z = "wall" bounds z by two free-slip walls
    through the first and last planes (z spacing lz / (nz - 1))."""

    def __init__(self, shape, lengths=(2 * np.pi,) * 3, cs=1.0, nu=5e-3, precision="fp64",
                 form="55p", entropy_mode=1, device=None, stream=None, bc_z="periodic"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("gbfd needs a CUDA device; there is no CPU path")
        self.torch = torch
        self.device = torch.device(device or "cuda")
        self.params = make_params(shape, lengths, cs, nu, precision, form, entropy_mode, bc_z)
        self.shape = tuple(shape)
        self.nfields = 5 if entropy_mode else 4
        nbytes = gbfd_workspace_bytes(self.params)
        if nbytes == 0:
            raise GbfdError(1, "invalid parameters")
        self.stream = stream or torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.ctx = gbfd_init(self.params, self.workspace.data_ptr(), nbytes,
                             self.stream.cuda_stream)

    def close(self):
        if getattr(self, "ctx", None):
            gbfd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_option(self, key, value):
        gbfd_set_option(self.ctx, key, value)

    def set_state(self, state):
        """state: numpy (host) or torch (host or device) array, float64 or float32."""
        torch = self.torch
        if isinstance(state, np.ndarray):
            state = torch.from_numpy(np.ascontiguousarray(state))
        assert tuple(state.shape) == (self.nfields,) + self.shape, state.shape
        state = state.contiguous()
        is64 = state.dtype == torch.float64
        if not is64 and state.dtype != torch.float32:
            raise TypeError("state must be float64 or float32")
        gbfd_set_state(self.ctx, state.data_ptr(), state.is_cuda, is64)
        if not state.is_cuda:
            self.stream.synchronize()  # the host buffer may be released after return

    def get_state(self, fp64=True, out=None):
        """Returns a numpy array (host), or fills `out` (torch, host or device)."""
        torch = self.torch
        if out is None:
            out = np.empty((self.nfields,) + self.shape, dtype=np.float64 if fp64 else np.float32)
            gbfd_get_state(self.ctx, out.ctypes.data, 0, fp64)
            return out
        gbfd_get_state(self.ctx, out.data_ptr(), out.is_cuda, out.dtype == torch.float64)
        return out

    def rk3_step(self, dt, nsteps=1):
        gbfd_rk3_step(self.ctx, dt, nsteps)

    def rk3_step_forced(self, dt, f0, k, phi, e):
        """Forced RK3 steps (Sect. 6): one step per entry of phi."""
        gbfd_rk3_step_forced(self.ctx, dt, f0, k, phi, e)

    def substep(self, s, dt):
        gbfd_substep(self.ctx, s, dt)

    def diagnostics(self):
        return gbfd_diagnostics(self.ctx).as_dict()

    def cfl_dt(self, cfl=0.4, cnu=0.25):
        return gbfd_cfl_dt(self.ctx, cfl, cnu)

    def sync(self):
        gbfd_sync(self.ctx)

    def launches(self):
        return gbfd_launch_count(self.ctx)

    def autotune(self, reps=3, cache_path=None):
        return gbfd_autotune(self.ctx, reps, cache_path)


# ------------------------------------------------------------ batched form

def _bcheck(status, b=None):
    if status != GBFD_OK:
        raise GbfdError(status, load().gbfd_batch_last_error(b).decode(errors="replace"))


class Batch:
    """Many independent periodic cubic boxes (FP32, 55-point) advanced by one
    persistent launch per substep, replayed from a CUDA graph.

    n, lengths, nu: per-box points per side, side length and viscosity."""

    def __init__(self, n, lengths, nu, cs=1.0, entropy_mode=1, device=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("gbfd needs a CUDA device; there is no CPU path")
        L = load()
        self.torch = torch
        self.n = [int(v) for v in n]
        self.nbox = len(self.n)
        self.nfields = 5 if entropy_mode else 4
        self._n = (ctypes.c_int32 * self.nbox)(*self.n)
        self._len = (ctypes.c_double * self.nbox)(*[float(v) for v in lengths])
        self._nu = (ctypes.c_double * self.nbox)(*[float(v) for v in nu])
        nbytes = L.gbfd_batch_workspace_bytes(self.nbox, self._n, int(entropy_mode))
        if nbytes == 0:
            raise GbfdError(1, "invalid batch sizes")
        self.device = torch.device(device or "cuda")
        self.stream = stream or torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.b = _VP()
        _bcheck(L.gbfd_batch_init(self.nbox, self._n, self._len, self._nu, float(cs),
                                  int(entropy_mode), _VP(self.workspace.data_ptr()), nbytes,
                                  _VP(self.stream.cuda_stream), ctypes.byref(self.b)))

    def close(self):
        if getattr(self, "b", None):
            load().gbfd_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_state(self, box, state):
        torch = self.torch
        if isinstance(state, np.ndarray):
            state = torch.from_numpy(np.ascontiguousarray(state))
        state = state.contiguous()
        n = self.n[box]
        assert tuple(state.shape) == (self.nfields, n, n, n), state.shape
        _bcheck(load().gbfd_batch_set_state(self.b, int(box), _VP(state.data_ptr()),
                                            int(state.is_cuda),
                                            int(state.dtype == torch.float64)), self.b)

    def get_state(self, box, fp64=True):
        n = self.n[box]
        out = np.empty((self.nfields, n, n, n), dtype=np.float64 if fp64 else np.float32)
        _bcheck(load().gbfd_batch_get_state(self.b, int(box), _VP(out.ctypes.data), 0, int(fp64)),
                self.b)
        return out

    def step(self, dt, nsteps=1):
        arr = (ctypes.c_double * self.nbox)(*[float(v) for v in dt])
        _bcheck(load().gbfd_batch_step(self.b, arr, int(nsteps)), self.b)

    def diagnostics(self, box):
        d = gbfd_diag()
        _bcheck(load().gbfd_batch_diagnostics(self.b, int(box), ctypes.byref(d)), self.b)
        return d.as_dict()

    def sync(self):
        _bcheck(load().gbfd_batch_sync(self.b), self.b)

    def set_option(self, key, value):
        _bcheck(load().gbfd_batch_set_option(self.b, int(key), int(value)), self.b)

    def get_option(self, key):
        v = ctypes.c_int64()
        _bcheck(load().gbfd_batch_get_option(self.b, int(key), ctypes.byref(v)), self.b)
        return v.value

    def autotune(self, steps=2):
        zc = ctypes.c_int()
        ms = ctypes.c_double()
        _bcheck(load().gbfd_batch_autotune(self.b, int(steps), ctypes.byref(zc), ctypes.byref(ms)),
                self.b)
        return zc.value, ms.value

    def launches(self):
        return load().gbfd_batch_launch_count(self.b)


# ------------------------------------------------------------ correction network

def _ccheck(status, c=None):
    if status != GBFD_OK:
        raise GbfdError(status, load().gbfd_cnn_last_error(c).decode(errors="replace"))


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class CNN:
    """The coarse-grid correction network (see include/gbfd.h) on an n^3 grid,
    training on up to `batch` samples at a time.  State tensors are torch
    CUDA float32 [batch, 5, n, n, n]."""

    def __init__(self, n, batch=1, device=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("gbfd needs a CUDA device; there is no CPU path")
        L = load()
        self.torch = torch
        self.n = int(n)
        self.batch = int(batch)
        nbytes = L.gbfd_cnn_workspace_bytes(self.n, self.batch)
        if nbytes == 0:
            raise GbfdError(1, "invalid network grid / batch")
        self.device = torch.device(device or "cuda")
        self.stream = stream or torch.cuda.current_stream(self.device)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes + 1024, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 1023) // 1024 * 1024
        self.c = _VP()
        _ccheck(L.gbfd_cnn_init(self.n, self.batch, _VP(aligned), nbytes,
                                _VP(self.stream.cuda_stream), ctypes.byref(self.c)))
        self.nparams = L.gbfd_cnn_param_count()

    def close(self):
        if getattr(self, "c", None):
            load().gbfd_cnn_destroy(self.c)
            self.c = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def flatten(p):
        """Oracle-style dict {W1,b1,W2,b2,W3,b3} -> ABI parameter vector."""
        return np.concatenate([np.asarray(p[k], dtype=np.float64).ravel()
                               for k in ("W1", "b1", "W2", "b2", "W3", "b3")]).astype(np.float32)

    @staticmethod
    def unflatten(v, hidden=32, cin=5, cout=5):
        shapes = [("W1", (hidden, cin, 3, 3, 3)), ("b1", (hidden,)),
                  ("W2", (hidden, hidden, 3, 3, 3)), ("b2", (hidden,)),
                  ("W3", (cout, hidden, 3, 3, 3)), ("b3", (cout,))]
        out, i = {}, 0
        for k, sh in shapes:
            m = int(np.prod(sh))
            out[k] = np.asarray(v[i:i + m], dtype=np.float64).reshape(sh)
            i += m
        return out

    def set_option(self, key, value):
        """GBFD_CNN_OPT_CONV_GRID / GBFD_CNN_OPT_WGRAD_PARTS (launch shapes)."""
        _ccheck(load().gbfd_cnn_set_option(self.c, int(key), ctypes.c_int64(int(value))), self.c)

    def set_params(self, p):
        v = np.ascontiguousarray(p if isinstance(p, np.ndarray) else self.flatten(p),
                                 dtype=np.float32)
        assert v.size == self.nparams
        _ccheck(load().gbfd_cnn_set_params(self.c, _fptr(v)), self.c)

    def get_params(self):
        v = np.empty(self.nparams, dtype=np.float32)
        _ccheck(load().gbfd_cnn_get_params(self.c, _fptr(v)), self.c)
        return v

    def set_norm(self, mean_in, std_in, std_out):
        a = [np.ascontiguousarray(x, dtype=np.float32) for x in (mean_in, std_in, std_out)]
        _ccheck(load().gbfd_cnn_set_norm(self.c, *[_fptr(x) for x in a]), self.c)

    def _dev(self, x):
        x = x.contiguous()
        assert x.is_cuda and x.dtype == self.torch.float32 and x.shape[1] == 5
        return x

    def forward(self, xs, nf=5):
        xs = self._dev(xs)
        ys = self.torch.empty_like(xs)
        _ccheck(load().gbfd_cnn_forward(self.c, _VP(xs.data_ptr()), nf, xs.shape[0],
                                        _VP(ys.data_ptr())), self.c)
        return ys

    def gradients(self, xs, ts, nf=5):
        xs, ts = self._dev(xs), self._dev(ts)
        g = np.empty(self.nparams, dtype=np.float32)
        loss = ctypes.c_double()
        _ccheck(load().gbfd_cnn_gradients(self.c, _VP(xs.data_ptr()), _VP(ts.data_ptr()), nf,
                                          xs.shape[0], _fptr(g), ctypes.byref(loss)), self.c)
        return g, loss.value

    def train_step(self, xs, ts, lr, nf=5, want_loss=True):
        xs, ts = self._dev(xs), self._dev(ts)
        loss = ctypes.c_double()
        _ccheck(load().gbfd_cnn_train_step(self.c, _VP(xs.data_ptr()), _VP(ts.data_ptr()), nf,
                                           xs.shape[0], float(lr),
                                           ctypes.byref(loss) if want_loss else None), self.c)
        return loss.value if want_loss else None

    def apply(self, solver):
        _ccheck(load().gbfd_cnn_apply(self.c, solver.ctx), self.c)

    def step_corrected(self, solver, dt, nsteps=1):
        _ccheck(load().gbfd_step_corrected(solver.ctx, self.c, float(dt), int(nsteps)), self.c)

    def launches(self):
        return load().gbfd_cnn_launch_count(self.c)


def box_filter(solver, r=4):
    """Centred box filter of a cubic FP32 solver's state to an r times coarser
    grid; returns a torch CUDA float32 tensor [nf, nc, nc, nc]."""
    torch = solver.torch
    n = solver.shape[0]
    out = torch.empty((solver.nfields, n // r, n // r, n // r), dtype=torch.float32,
                      device=solver.device)
    st = load().gbfd_box_filter(solver.ctx, int(r), _VP(out.data_ptr()))
    if st != GBFD_OK:
        raise GbfdError(st, "box filter needs a cubic FP32 context with n % r == 0")
    return out
