"""Python binding of the FP64 CPU oracle (``lsh_oracle.c``).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow restatement of the
Galerkin-discretised Lippmann-Schwinger equation of Brisard & Legoll
(arXiv:1411.0330, Sec. 3, Eq. (13)) used to check the CUDA path.  Only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference
leg of ``bench.py`` may import it.  It imports nothing from the product
package and the product package imports nothing from here.

Fields are numpy arrays of shape ``(c, n2, n1, n0)`` (3D) or ``(c, n1, n0)``
(2D), axis 0 fastest in memory, Mandel components for elasticity.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lsh_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liblsh_oracle.so")

SCALAR, ELASTIC = 0, 1
TRUNCATED, FILTERED, FINITE_DIFF, CONSISTENT = 0, 1, 2, 3
SOLVER_AUTO, SOLVER_CG, SOLVER_MINRES = 0, 1, 2
_STATUS = {0: "ok", 1: "invalid argument", 2: "A_beta - A0 singular", 3: "A0 not SPD",
           4: "breakdown", 5: "not converged", 6: "problem too large", 7: "out of memory"}

_lock = threading.Lock()
_lib = None


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what}: {_STATUS.get(code, code)}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available).  Returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                              os.path.getmtime(os.path.join(_HERE, "lsh_oracle.h")))):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
            _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Problem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("physics", ctypes.c_int),
                ("green", ctypes.c_int), ("nphase", ctypes.c_int),
                ("phase_moduli", ctypes.POINTER(ctypes.c_double)),
                ("ref_moduli", ctypes.POINTER(ctypes.c_double)),
                ("phase", ctypes.POINTER(ctypes.c_ubyte)),
                ("scale", ctypes.POINTER(ctypes.c_double)),
                ("frac", ctypes.POINTER(ctypes.c_double))]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Problem)
            dp = ctypes.POINTER(ctypes.c_double)
            lib.or_ncomp.argtypes = [P]
            lib.or_nvox.argtypes = [P]
            lib.or_nvox.restype = ctypes.c_long
            lib.or_default_reference.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
            lib.or_local_operator.argtypes = [P, dp, ctypes.POINTER(ctypes.c_ubyte)]
            lib.or_gamma0.argtypes = [P, dp, dp]
            lib.or_gamma0.restype = None
            lib.or_gamma_hat.argtypes = [P, ctypes.POINTER(ctypes.c_int), dp]
            lib.or_gamma_hat.restype = None
            lib.or_dft.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, dp]
            lib.or_dft.restype = None
            lib.or_dft_naive.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, dp, dp]
            lib.or_dft_naive.restype = None
            lib.or_apply.argtypes = [P, dp, dp]
            lib.or_solve.argtypes = [P, dp, dp, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp]
            lib.or_dense_solve.argtypes = [P, dp, dp]
            lib.or_effective.argtypes = [P, ctypes.c_double, ctypes.c_int, ctypes.c_int, dp, dp, dp]
            lib.or_effective_variational.argtypes = [P, dp, dp]
            lib.or_scale_gradient.argtypes = [P, dp, dp, dp]
            _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Problem:
    """Inputs of one corrector problem (Sec. 2.2 / Sec. 3).

    phase: uint8 array of shape (n2, n1, n0) or (n1, n0), phase id per voxel.
    phase_moduli: scalar -> (nphase, d, d) symmetric matrices; elastic ->
        (nphase, 2) rows of (bulk K, shear mu).
    ref: reference medium in the same format as one phase; None -> the
        oracle's default rule (half the softest phase).
    scale: optional per-voxel factor s with A_beta = s_beta A_phase(beta).
    frac: optional per-voxel volume fraction of phase 1 (two phases): the local
        operator becomes the voxel average of (A - A0)^{-1}, Eq. (def_ah).
    """

    def __init__(self, phase, phase_moduli, physics=SCALAR, green=TRUNCATED, ref=None, scale=None, frac=None):
        phase = np.ascontiguousarray(phase, dtype=np.uint8)
        self.dim = phase.ndim
        if self.dim not in (2, 3):
            raise ValueError("phase must be 2D or 3D")
        self.shape = phase.shape
        self.n = tuple(reversed(phase.shape))  # (n0, n1[, n2])
        self.physics = physics
        self.green = green
        self.phase = phase
        self.phase_moduli = np.ascontiguousarray(phase_moduli, dtype=np.float64)
        self.nphase = self.phase_moduli.shape[0]
        if ref is None:
            ref = default_reference(self.dim, physics, self.phase_moduli)
        self.ref = np.ascontiguousarray(ref, dtype=np.float64)
        self.scale = None if scale is None else np.ascontiguousarray(scale, dtype=np.float64)
        self.frac = None if frac is None else np.ascontiguousarray(frac, dtype=np.float64)
        self.c = 6 if physics == ELASTIC else self.dim
        self.V = int(phase.size)

    @property
    def field_shape(self):
        return (self.c,) + self.shape

    def _struct(self) -> _Problem:
        s = _Problem()
        s.dim = self.dim
        n = list(self.n) + [1] * (3 - len(self.n))
        s.n = (ctypes.c_int * 3)(*n)
        s.physics, s.green, s.nphase = self.physics, self.green, self.nphase
        s.phase_moduli = _dptr(self.phase_moduli)
        s.ref_moduli = _dptr(self.ref)
        s.phase = self.phase.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
        s.scale = _dptr(self.scale) if self.scale is not None else ctypes.POINTER(ctypes.c_double)()
        s.frac = _dptr(self.frac) if self.frac is not None else ctypes.POINTER(ctypes.c_double)()
        return s

    def with_(self, **kw) -> "Problem":
        args = dict(phase=self.phase, phase_moduli=self.phase_moduli, physics=self.physics,
                    green=self.green, ref=self.ref, scale=self.scale, frac=self.frac)
        args.update(kw)
        return Problem(**args)


def _check(code: int, what: str):
    if code != 0:
        raise OracleError(code, what)


def default_reference(dim: int, physics: int, phase_moduli) -> np.ndarray:
    lib = _load()
    pm = np.ascontiguousarray(phase_moduli, dtype=np.float64)
    out = np.zeros(2 if physics == ELASTIC else dim * dim)
    _check(lib.or_default_reference(dim, physics, pm.shape[0], _dptr(pm), _dptr(out)), "default_reference")
    return out if physics == ELASTIC else out.reshape(dim, dim)


def local_operator(prob: Problem):
    lib = _load()
    s = prob._struct()
    M = np.zeros((prob.V, prob.c, prob.c))
    act = np.zeros(prob.V, dtype=np.uint8)
    _check(lib.or_local_operator(ctypes.byref(s), _dptr(M),
                                 act.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))), "local_operator")
    return M, act.reshape(prob.shape)


def gamma0(prob: Problem, xi) -> np.ndarray:
    lib = _load()
    s = prob._struct()
    x = np.zeros(3)
    x[:len(xi)] = xi
    G = np.zeros(prob.c * prob.c)
    lib.or_gamma0(ctypes.byref(s), _dptr(x), _dptr(G))
    return G.reshape(prob.c, prob.c)


def gamma_hat(prob: Problem, k) -> np.ndarray:
    lib = _load()
    s = prob._struct()
    kk = (ctypes.c_int * 3)(*(list(k) + [0] * (3 - len(k))))
    G = np.zeros(2 * prob.c * prob.c)
    lib.or_gamma_hat(ctypes.byref(s), kk, _dptr(G))
    return (G[0::2] + 1j * G[1::2]).reshape(prob.c, prob.c)


def dft(a: np.ndarray, sign: int = -1, naive: bool = False) -> np.ndarray:
    """Unnormalised DFT of a complex 2D/3D array (numpy axis order (n2, n1, n0))."""
    lib = _load()
    a = np.ascontiguousarray(a, dtype=np.complex128)
    dim = a.ndim
    n = (ctypes.c_int * 3)(*(list(reversed(a.shape)) + [1] * (3 - dim)))
    buf = a.view(np.float64).copy()
    if naive:
        out = np.zeros_like(buf)
        lib.or_dft_naive(dim, n, sign, _dptr(buf), _dptr(out))
        return out.view(np.complex128).reshape(a.shape)
    lib.or_dft(dim, n, sign, _dptr(buf))
    return buf.view(np.complex128).reshape(a.shape)


def apply(prob: Problem, x: np.ndarray) -> np.ndarray:
    lib = _load()
    s = prob._struct()
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(prob.field_shape)
    y = np.zeros_like(x)
    _check(lib.or_apply(ctypes.byref(s), _dptr(x), _dptr(y)), "apply")
    return y


def solve(prob: Problem, load, tol=1e-12, maxit=10000, solver=SOLVER_AUTO):
    """Returns (tau, iterations, relative residual)."""
    lib = _load()
    s = prob._struct()
    ld = np.ascontiguousarray(load, dtype=np.float64)
    tau = np.zeros(prob.field_shape)
    info = np.zeros(2)
    _check(lib.or_solve(ctypes.byref(s), _dptr(ld), _dptr(tau), tol, maxit, solver, _dptr(info)), "solve")
    return tau, int(info[0]), float(info[1])


def dense_solve(prob: Problem, load) -> np.ndarray:
    lib = _load()
    s = prob._struct()
    ld = np.ascontiguousarray(load, dtype=np.float64)
    tau = np.zeros(prob.field_shape)
    _check(lib.or_dense_solve(ctypes.byref(s), _dptr(ld), _dptr(tau)), "dense_solve")
    return tau


def effective(prob: Problem, tol=1e-12, maxit=10000, solver=SOLVER_AUTO, return_tau=False):
    """A*_h (c x c, Astar[i, j] = e_i . A*_h e_j) and per-load (iterations, relres)."""
    lib = _load()
    s = prob._struct()
    A = np.zeros(prob.c * prob.c)
    info = np.zeros(2 * prob.c)
    tau_all = np.zeros((prob.c,) + prob.field_shape) if return_tau else None
    tp = _dptr(tau_all) if return_tau else ctypes.POINTER(ctypes.c_double)()
    _check(lib.or_effective(ctypes.byref(s), tol, maxit, solver, _dptr(A), tp, _dptr(info)), "effective")
    out = (A.reshape(prob.c, prob.c), info.reshape(prob.c, 2))
    return out + (tau_all,) if return_tau else out


def effective_variational(prob: Problem, tau_all: np.ndarray) -> np.ndarray:
    lib = _load()
    s = prob._struct()
    t = np.ascontiguousarray(tau_all, dtype=np.float64)
    A = np.zeros(prob.c * prob.c)
    _check(lib.or_effective_variational(ctypes.byref(s), _dptr(t), _dptr(A)), "effective_variational")
    return A.reshape(prob.c, prob.c)


def scale_gradient(prob: Problem, tau_all: np.ndarray, W) -> np.ndarray:
    lib = _load()
    s = prob._struct()
    t = np.ascontiguousarray(tau_all, dtype=np.float64)
    w = np.ascontiguousarray(W, dtype=np.float64)
    g = np.zeros(prob.V)
    _check(lib.or_scale_gradient(ctypes.byref(s), _dptr(t), _dptr(w), _dptr(g)), "scale_gradient")
    return g.reshape(prob.shape)
