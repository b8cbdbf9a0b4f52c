"""ctypes binding of liblsh (include/lsh.h): argument marshalling only.

Every step of the Lippmann-Schwinger solve runs in the CUDA library; this
module only converts arguments, allocates the device workspace with torch
(PyTorch is used for device memory and streams) and turns status codes into
exceptions.  There is no CPU fallback: constructing a Handle raises if the
library cannot be loaded or CUDA is unavailable.

Field layout: torch tensors of shape (c, n2, n1, n0) (3D) or (c, n1, n0)
(2D), contiguous, on the handle's device; Mandel components for elasticity.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

SCALAR, ELASTIC = 0, 1
TRUNCATED, FILTERED, FD = 0, 1, 2
FP64, MIXED = 0, 1
F64, F32, F64_DF = 0, 1, 2
SOLVER_AUTO, SOLVER_CG, SOLVER_MINRES, SOLVER_BASIC, SOLVER_SYMMLQ = 0, 1, 2, 3, 4

OK, ERR_INVALID_ARG, ERR_UNSUPPORTED_SIZE, ERR_REFERENCE_INDEFINITE, ERR_SINGULAR_CONTRAST, \
    ERR_BREAKDOWN, ERR_NOT_CONVERGED, ERR_WORKSPACE, ERR_CUDA, ERR_UNSUPPORTED = range(10)

_lock = threading.Lock()
_lib = None


class LSHError(RuntimeError):
    def __init__(self, status: int, what: str):
        msg = _lib.lsh_status_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{what}: {msg} (status {status})")
        self.status = status


class _Problem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("physics", ctypes.c_int),
                ("green", ctypes.c_int), ("precision", ctypes.c_int), ("nphase", ctypes.c_int),
                ("phase_moduli", ctypes.POINTER(ctypes.c_double)),
                ("ref_moduli", ctypes.POINTER(ctypes.c_double)),
                ("phase", ctypes.c_void_p), ("phase_on_host", ctypes.c_int),
                ("scale", ctypes.c_void_p), ("nbatch", ctypes.c_int), ("max_systems", ctypes.c_int),
                ("scale_kind", ctypes.c_int)]


class _Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("maxit", ctypes.c_int), ("solver", ctypes.c_int),
                ("inner_tol", ctypes.c_double), ("max_outer", ctypes.c_int), ("check_every", ctypes.c_int),
                ("warm_start", ctypes.c_int), ("no_graphs", ctypes.c_int)]


class _TuneReport(ctypes.Structure):
    _fields_ = [("xf_variant", ctypes.c_int), ("x_variant", ctypes.c_int), ("y_variant", ctypes.c_int),
                ("z_variant", ctypes.c_int), ("xf_ms", ctypes.c_float * 2), ("x_ms", ctypes.c_float * 4),
                ("y_ms", ctypes.c_float * 2), ("z_ms", ctypes.c_float * 10), ("xy_ms", ctypes.c_float * 2),
                ("zp_ms", ctypes.c_float * 7)]


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer", ctypes.c_int), ("applies64", ctypes.c_int),
                ("status", ctypes.c_int), ("relres", ctypes.c_double)]

    def as_dict(self):
        return {"iters": self.iters, "outer": self.outer, "applies64": self.applies64,
                "status": self.status, "relres": self.relres}


class _Profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("timed_iters", ctypes.c_longlong),
                ("pass_ms", ctypes.c_double * 6), ("pass_launches", ctypes.c_longlong * 6),
                ("timed_sys_iters", ctypes.c_longlong)]


PASS_NAMES = ["x_forward", "y_forward", "z_gamma", "y_inverse", "x_inverse_local", "cg_update"]

EXPORTS = ["lsh_workspace_size", "lsh_setup", "lsh_set_microstructure", "lsh_apply", "lsh_solve",
           "lsh_effective", "lsh_effective_grad", "lsh_profile_enable", "lsh_profile_read", "lsh_destroy",
           "lsh_status_string", "lsh_apply_noalloc", "lsh_effective_batch", "lsh_autotune",
           "lsh_set_variants", "lsh_check_bounded_wait"]


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = True):
    """Load liblsh.so (building it with nvcc if it is missing and allowed)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path):
                if not build_if_missing:
                    raise OSError(f"liblsh.so not built ({path})")
                _build.build()
            lib = ctypes.CDLL(path)
            P = ctypes.POINTER(_Problem)
            vp = ctypes.c_void_p
            dp = ctypes.POINTER(ctypes.c_double)
            lib.lsh_status_string.restype = ctypes.c_char_p
            lib.lsh_status_string.argtypes = [ctypes.c_int]
            lib.lsh_workspace_size.argtypes = [P, ctypes.POINTER(ctypes.c_size_t)]
            lib.lsh_setup.argtypes = [P, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
            lib.lsh_set_microstructure.argtypes = [vp, vp, vp, ctypes.c_int]
            lib.lsh_apply.argtypes = [vp, ctypes.c_int, vp, vp]
            lib.lsh_solve.argtypes = [vp, dp, vp, ctypes.POINTER(_Opts), ctypes.POINTER(_Info)]
            lib.lsh_effective.argtypes = [vp, ctypes.POINTER(_Opts), dp, vp, ctypes.POINTER(_Info)]
            lib.lsh_effective_grad.argtypes = [vp, vp, dp, vp]
            lib.lsh_profile_enable.argtypes = [vp, ctypes.c_int]
            lib.lsh_profile_read.argtypes = [vp, ctypes.POINTER(_Profile), ctypes.c_int]
            lib.lsh_destroy.argtypes = [vp]
            lib.lsh_destroy.restype = None
            lib.lsh_apply_noalloc.argtypes = [P, vp, vp, vp]
            lib.lsh_autotune.argtypes = [vp, ctypes.POINTER(_TuneReport)]
            lib.lsh_set_variants.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.lsh_check_bounded_wait.argtypes = [vp, ctypes.c_double]
            lib.lsh_effective_batch.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(_Opts), dp,
                                                ctypes.POINTER(_Info)]
            _lib = lib
    return _lib


def _check(status: int, what: str, allow=()):
    if status != OK and status not in allow:
        raise LSHError(status, what)
    return status


def _problem_struct(phase_ptr, on_host, shape, physics, green, precision, moduli, ref, scale_ptr, nbatch=1,
                    max_systems=0, scale_kind=0):
    s = _Problem()
    dim = len(shape)
    s.dim = dim
    n = list(reversed(shape)) + [1] * (3 - dim)
    s.n = (ctypes.c_int * 3)(*n)
    s.physics, s.green, s.precision = physics, green, precision
    s.nphase = moduli.shape[0]
    s.phase_moduli = moduli.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    s.ref_moduli = ref.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if ref is not None else \
        ctypes.POINTER(ctypes.c_double)()
    s.phase = phase_ptr
    s.phase_on_host = 1 if on_host else 0
    s.scale = scale_ptr
    s.nbatch = nbatch
    s.max_systems = max_systems
    s.scale_kind = scale_kind
    return s


def _opts(tol, maxit, solver, inner_tol, max_outer, check_every, warm_start=False, graphs=True):
    return _Opts(tol, maxit, solver, inner_tol, max_outer, check_every, 1 if warm_start else 0,
                 0 if graphs else 1)


def workspace_size(shape, phase_moduli, physics=SCALAR, green=TRUNCATED, precision=FP64, ref=None,
                   has_scale=False, nbatch=1, max_systems=0) -> int:
    """Workspace bytes for a problem (host-only computation; no GPU needed)."""
    lib = load_library()
    mods = np.ascontiguousarray(phase_moduli, dtype=np.float64)
    refa = None if ref is None else np.ascontiguousarray(ref, dtype=np.float64)
    dummy = ctypes.c_void_p(1)
    s = _problem_struct(dummy, True, tuple(shape), physics, green, precision, mods, refa,
                        ctypes.c_void_p(1) if has_scale else None, nbatch, max_systems)
    out = ctypes.c_size_t(0)
    _check(lib.lsh_workspace_size(ctypes.byref(s), ctypes.byref(out)), "lsh_workspace_size")
    return out.value


def apply_noalloc(phase, x, phase_moduli, physics=SCALAR, green=TRUNCATED, ref=None, scale=None, out=None,
                  stream=None):
    """y = K x through lsh_apply_noalloc: no handle, no workspace, nothing allocated by
    the library (its scratch is a fixed 64 MiB device array).  phase, scale, x are CUDA
    tensors of one microstructure; returns y (float64, like x)."""
    import torch
    lib = load_library()
    phase = phase.contiguous()
    x = x.to(torch.float64).contiguous()
    y = out if out is not None else torch.empty_like(x)
    mods = np.ascontiguousarray(phase_moduli, dtype=np.float64)
    refa = None if ref is None else np.ascontiguousarray(ref, dtype=np.float64)
    sc = None if scale is None else scale.to(torch.float32).contiguous()
    s = _problem_struct(ctypes.c_void_p(phase.data_ptr()), False, tuple(phase.shape), physics, green, FP64, mods,
                        refa, ctypes.c_void_p(sc.data_ptr()) if sc is not None else None)
    st = stream if stream is not None else torch.cuda.current_stream(x.device)
    _check(lib.lsh_apply_noalloc(ctypes.byref(s), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                 ctypes.c_void_p(st.cuda_stream)), "lsh_apply_noalloc")
    return y


class Handle:
    """One corrector problem on one GPU (Sec. 2.2 / Sec. 3 of the paper).

    phase: uint8 torch tensor (device or CPU) or numpy array, shape (n2, n1, n0) or (n1, n0);
        with batch=True a leading axis stacks microstructures of the same grid.
    phase_moduli: scalar -> (nphase, d, d) diagonal conductivities; elastic -> (nphase, 2) (K, mu).
    ref: reference medium in the same format as one phase, or None (half the softest phase).
    scale: optional per-voxel float32 factor s (A_beta = s_beta A_phase), shaped like phase.
    fraction: instead of scale, the per-voxel volume fraction of phase 1 of a two-phase medium
        (sub-voxel averaging of (A - A0)^{-1}, Eq. (def_ah)); the phase map is then not used.
    max_systems: systems (microstructure x load) solved at once; bounds the workspace.
    tune: run lsh_autotune after setup (times the FP32 y / z pass variants, keeps the fastest).
    """

    def __init__(self, phase, phase_moduli, physics=SCALAR, green=TRUNCATED, precision=FP64, ref=None,
                 scale=None, device=None, stream=None, batch=False, max_systems=0, tune=False, fraction=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("liblsh needs a CUDA device; no CPU fallback exists")
        self._torch = torch
        self.lib = load_library()
        self.device = torch.device(device if device is not None else "cuda", )
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._own_stream = self.stream != torch.cuda.current_stream(self.device)
        if isinstance(phase, np.ndarray):
            phase_t = torch.from_numpy(np.ascontiguousarray(phase, dtype=np.uint8))
        else:
            phase_t = phase.contiguous()
            if phase_t.dtype != torch.uint8:
                raise TypeError("phase must be uint8")
        self.batch = bool(batch)
        self.nbatch = int(phase_t.shape[0]) if batch else 1
        self.shape = tuple(phase_t.shape[1:]) if batch else tuple(phase_t.shape)
        self.dim = len(self.shape)
        self.physics = physics
        self.precision = precision
        self.c = 6 if physics == ELASTIC else self.dim
        self.V = int(np.prod(self.shape))
        self.moduli = np.ascontiguousarray(phase_moduli, dtype=np.float64)
        self.scale_kind = 0
        if fraction is not None:
            if scale is not None:
                raise ValueError("scale and fraction are exclusive")
            scale, self.scale_kind = fraction, 1
        self.ref = None if ref is None else np.ascontiguousarray(ref, dtype=np.float64)
        on_host = phase_t.device.type == "cpu"
        scale_t = None
        if scale is not None:
            scale_t = torch.as_tensor(scale, dtype=torch.float32)
            scale_t = scale_t.contiguous() if not on_host else scale_t.cpu().contiguous()
            if not on_host:
                scale_t = scale_t.to(self.device)
        self.has_scale = scale_t is not None
        self.phase_source = phase_t  # kept so the scale field can be replaced alone
        s = _problem_struct(ctypes.c_void_p(phase_t.data_ptr()), on_host, self.shape, physics, green, precision,
                            self.moduli, self.ref, ctypes.c_void_p(scale_t.data_ptr()) if scale_t is not None else None,
                            self.nbatch, max_systems, self.scale_kind)
        nbytes = ctypes.c_size_t(0)
        _check(self.lib.lsh_workspace_size(ctypes.byref(s), ctypes.byref(nbytes)), "lsh_workspace_size")
        self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        self._wait_inputs()
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(self.lib.lsh_setup(ctypes.byref(s), ctypes.c_void_p(self.workspace.data_ptr()), nbytes.value,
                                      ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)), "lsh_setup")
        self._h = h
        self.tune_report = self.autotune() if tune else None

    # ------------------------------------------------------------------ helpers
    @property
    def field_shape(self):
        return ((self.nbatch,) if self.batch else ()) + (self.c,) + self.shape

    @property
    def grid_shape(self):
        return ((self.nbatch,) if self.batch else ()) + self.shape

    def _field(self, x, dtype):
        t = self._torch
        if not isinstance(x, t.Tensor):
            x = t.as_tensor(np.asarray(x), dtype=dtype)
        x = x.to(device=self.device, dtype=dtype).contiguous()
        if tuple(x.shape) != self.field_shape:
            x = x.reshape(self.field_shape)
        return x

    def _wait_inputs(self):
        """With a stream of its own, the handle waits for work queued on the
        caller's current stream (its inputs) before using them."""
        if self._own_stream:
            self.stream.wait_stream(self._torch.cuda.current_stream(self.device))

    def _release_outputs(self):
        if self._own_stream:
            self._torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def close(self):
        if getattr(self, "_h", None):
            self.lib.lsh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ API
    def set_microstructure(self, phase, scale=None):
        t = self._torch
        if isinstance(phase, np.ndarray):
            phase = t.from_numpy(np.ascontiguousarray(phase, dtype=np.uint8))
        on_host = phase.device.type == "cpu"
        phase = phase.contiguous()
        sp = None
        if scale is not None:
            scale = t.as_tensor(scale, dtype=t.float32)
            scale = scale.cpu().contiguous() if on_host else scale.to(self.device).contiguous()
            sp = ctypes.c_void_p(scale.data_ptr())
        self._wait_inputs()
        _check(self.lib.lsh_set_microstructure(self._h, ctypes.c_void_p(phase.data_ptr()), sp, 1 if on_host else 0),
               "lsh_set_microstructure")

    def apply(self, x, out=None, dtype=None, double_float=False):
        """y = K x, the operator of Eq. (13) with the projection on I0.
        double_float=True (FP64 fields, mixed handles): evaluated in double-float
        arithmetic on the FP32 pipes, as the mixed solver's refinement residual is."""
        t = self._torch
        dtype = dtype or (x.dtype if isinstance(x, t.Tensor) and x.dtype in (t.float32, t.float64) else t.float64)
        x = self._field(x, dtype)
        y = out if out is not None else t.empty_like(x)
        self._wait_inputs()
        code = F32 if dtype != t.float64 else (F64_DF if double_float else F64)
        _check(self.lib.lsh_apply(self._h, code, ctypes.c_void_p(x.data_ptr()),
                                  ctypes.c_void_p(y.data_ptr())), "lsh_apply")
        self._release_outputs()
        return y

    def solve(self, load, tau=None, tol=1e-10, maxit=10000, solver=SOLVER_AUTO, inner_tol=0.0, max_outer=0,
              check_every=0, warm_start=False, raise_on_fail=True, graphs=True):
        """Solve Eq. (13) for the macroscopic load p (c values).  Returns (tau, info dict).
        graphs=False launches the CG kernels one by one instead of replaying a CUDA graph."""
        t = self._torch
        ld = np.ascontiguousarray(load, dtype=np.float64)
        if tau is None:
            tau = t.zeros(self.field_shape, dtype=t.float64, device=self.device)
        infos = (_Info * self.nbatch)()
        o = _opts(tol, maxit, solver, inner_tol, max_outer, check_every, warm_start, graphs)
        self._wait_inputs()
        st = self.lib.lsh_solve(self._h, ld.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                ctypes.c_void_p(tau.data_ptr()), ctypes.byref(o), infos)
        _check(st, "lsh_solve", allow=() if raise_on_fail else (ERR_NOT_CONVERGED, ERR_BREAKDOWN))
        out = [i.as_dict() for i in infos]
        return tau, (out if self.batch else out[0])

    def effective(self, tol=1e-10, maxit=10000, solver=SOLVER_AUTO, inner_tol=0.0, max_outer=0, check_every=0,
                  return_tau=False, tau_out=None, raise_on_fail=True, graphs=True):
        """A*_h (c x c numpy, A[i, j] = e_i . A*_h e_j; (nbatch, c, c) for a batch) and
        per-system info dicts (load-major within each microstructure)."""
        t = self._torch
        A = np.zeros(self.nbatch * self.c * self.c)
        infos = (_Info * (self.nbatch * self.c))()
        tau_all = tau_out
        if return_tau and tau_all is None:
            lead = (self.nbatch,) if self.batch else ()
            tau_all = t.empty(lead + (self.c, self.c) + self.shape, dtype=t.float64, device=self.device)
        o = _opts(tol, maxit, solver, inner_tol, max_outer, check_every, graphs=graphs)
        self._wait_inputs()
        st = self.lib.lsh_effective(self._h, ctypes.byref(o), A.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    ctypes.c_void_p(tau_all.data_ptr()) if tau_all is not None else None, infos)
        _check(st, "lsh_effective", allow=() if raise_on_fail else (ERR_NOT_CONVERGED, ERR_BREAKDOWN))
        A = A.reshape(self.nbatch, self.c, self.c) if self.batch else A.reshape(self.c, self.c)
        out = (A, [i.as_dict() for i in infos])
        return out + (tau_all,) if tau_all is not None else out

    def autotune(self):
        """Time the FP32 y / z pass variants on this handle and keep the fastest."""
        r = _TuneReport()
        self._wait_inputs()
        _check(self.lib.lsh_autotune(self._h, ctypes.byref(r)), "lsh_autotune")
        self.tune_report = {"xf_variant": r.xf_variant, "x_variant": r.x_variant, "y_variant": r.y_variant,
                            "z_variant": r.z_variant, "xf_ms": list(r.xf_ms), "x_ms": list(r.x_ms),
                            "y_ms": list(r.y_ms), "z_ms": list(r.z_ms), "xy_ms": list(r.xy_ms),
                            "zp_ms": list(r.zp_ms)}
        return self.tune_report

    def set_variants(self, xf_variant, x_variant, y_variant, z_variant):
        """Force the FP32 forward x / inverse x / y / z pass variants (see lsh_tune_report;
        y_variant 2: the plane passes)."""
        _check(self.lib.lsh_set_variants(self._h, int(xf_variant), int(x_variant), int(y_variant), int(z_variant)),
               "lsh_set_variants")

    def profile_enable(self, enable=True, every=1):
        """Per-pass CUDA-event timing of the CG iterations; every=k times one
        chunk of iterations in k (the others run without event nodes)."""
        _check(self.lib.lsh_profile_enable(self._h, max(int(every), 1) if enable else 0), "lsh_profile_enable")

    def profile_read(self, reset=False):
        p = _Profile()
        _check(self.lib.lsh_profile_read(self._h, ctypes.byref(p), 1 if reset else 0), "lsh_profile_read")
        return {"launches": p.launches, "timed_iters": p.timed_iters,
                "pass_ms": {n: p.pass_ms[i] for i, n in enumerate(PASS_NAMES)},
                "pass_launches": {n: p.pass_launches[i] for i, n in enumerate(PASS_NAMES)},
                "timed_sys_iters": p.timed_sys_iters}

    def check_bounded_wait(self, seconds=0.05):
        """Run the give-up path of the bounded device waits on purpose (a barrier that
        expects two arrivals gets one); returns the status code: ERR_CUDA when the wait
        gave up and the fault word reached the host."""
        return int(self.lib.lsh_check_bounded_wait(self._h, float(seconds)))

    def effective_grad(self, tau_all, W, out=None):
        """d(sum_ij W_ij e_i.A*_h e_j)/d s_beta for the per-voxel scale field."""
        t = self._torch
        w = np.ascontiguousarray(W, dtype=np.float64)
        g = out if out is not None else t.empty(self.grid_shape, dtype=t.float64, device=self.device)
        self._wait_inputs()
        _check(self.lib.lsh_effective_grad(self._h, ctypes.c_void_p(tau_all.data_ptr()),
                                           w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           ctypes.c_void_p(g.data_ptr())), "lsh_effective_grad")
        return g


def effective_batch(handles, tol=1e-10, maxit=10000, solver=SOLVER_AUTO, inner_tol=0.0, max_outer=0, check_every=0,
                    raise_on_fail=True, graphs=True):
    """lsh_effective on several handles at once (one host thread and one stream
    per handle, so their kernels overlap).  Returns one A per handle (c x c, or
    (nbatch, c, c) for a batch handle) and one list of info dicts per handle."""
    handles = list(handles)
    if not handles:
        return [], []
    lib = handles[0].lib
    sizes = [h.nbatch * h.c * h.c for h in handles]
    nsys = [h.nbatch * h.c for h in handles]
    A = np.zeros(sum(sizes))
    infos = (_Info * sum(nsys))()
    for h in handles:
        h._wait_inputs()
    hs = (ctypes.c_void_p * len(handles))(*[h._h.value for h in handles])
    o = _opts(tol, maxit, solver, inner_tol, max_outer, check_every, graphs=graphs)
    st = lib.lsh_effective_batch(len(handles), hs, ctypes.byref(o), A.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 infos)
    _check(st, "lsh_effective_batch", allow=() if raise_on_fail else (ERR_NOT_CONVERGED, ERR_BREAKDOWN))
    outA, outI, a0, i0 = [], [], 0, 0
    for h, na, ns in zip(handles, sizes, nsys):
        blk = A[a0:a0 + na]
        outA.append(blk.reshape((h.nbatch, h.c, h.c)) if h.batch else blk.reshape((h.c, h.c)))
        outI.append([infos[i0 + k].as_dict() for k in range(ns)])
        a0 += na
        i0 += ns
    return outA, outI


class GridBatch:
    """Many microstructures of uneven grids (Sec. 5 computes one effective
    tensor per microstructure): one batch handle per distinct grid.

    phases: list of uint8 arrays / tensors (any grid each); the other arguments
    as for Handle.  stream=None gives every grid handle its own CUDA stream and
    effective() solves them together (lsh_effective_batch, one host thread per
    handle); with a stream, every handle issues its work on that one stream and
    effective() solves the grids one after the other.  effective() returns the
    effective tensors in input order."""

    def __init__(self, phases, phase_moduli, physics=ELASTIC, green=FILTERED, precision=MIXED, ref=None,
                 device=None, max_systems=0, tune=True, stream=None):
        import torch
        self._torch = torch
        groups = {}
        for i, ph in enumerate(phases):
            groups.setdefault(tuple(ph.shape), []).append(i)
        self.order = []
        self.handles = []
        self.streams = []
        self.shared = stream is not None
        for shape, idx in sorted(groups.items(), key=lambda kv: -int(np.prod(kv[0])) * len(kv[1])):
            if isinstance(phases[idx[0]], np.ndarray):
                stack = torch.from_numpy(np.stack([np.asarray(phases[i], dtype=np.uint8) for i in idx]))
            else:
                stack = torch.stack([phases[i] for i in idx])
            dev = torch.device(device if device is not None else "cuda")
            st = stream if stream is not None else torch.cuda.Stream(device=dev)
            self.streams.append(st)
            self.handles.append(Handle(stack.to(dev), phase_moduli, physics=physics, green=green,
                                       precision=precision, ref=ref, device=dev, stream=st, batch=True,
                                       max_systems=max_systems, tune=tune))
            self.order.append(idx)
        self.n = len(phases)

    def grid_stacks(self, phases):
        """The phase maps regrouped as the handles hold them: one (nbatch, *grid) uint8 array per handle."""
        return [np.stack([np.asarray(phases[i], dtype=np.uint8) for i in idx]) for idx in self.order]

    def set_microstructures(self, stacks):
        """Replace every handle's phase maps; stacks as grid_stacks() returns them (numpy, or CPU
        tensors -- pinned memory lets the copies run asynchronously -- or device tensors)."""
        for h, st in zip(self.handles, stacks):
            h.set_microstructure(st)

    def effective(self, **kw):
        if self.shared:
            res = [h.effective(**kw) for h in self.handles]
            As, Is = [r[0] for r in res], [r[1] for r in res]
        else:
            # the phase uploads ran on the handles' streams: wait for them before solving
            for st in self.streams:
                st.synchronize()
            As, Is = effective_batch(self.handles, **kw)
        A = [None] * self.n
        infos = [None] * self.n
        for idx, Ah, Ih, h in zip(self.order, As, Is, self.handles):
            for k, i in enumerate(idx):
                A[i] = Ah[k]
                infos[i] = Ih[k * h.c:(k + 1) * h.c]
        return A, infos

    def close(self):
        for h in self.handles:
            h.close()
