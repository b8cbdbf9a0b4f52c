"""lsh_apply_noalloc, the allocation-free operator application, against lsh_apply.

lsh_apply_noalloc serves callers that cannot allocate device memory where they
need K x (plugins inside host programs that own the device memory, processes
whose memory belongs to another framework's pool, code that must avoid the
synchronisation cudaMalloc / cudaFree may cause).  Its scratch is a fixed
array inside the library; this file checks, through the C ABI, that two calls
in a row give what the workspace-based lsh_apply gives, and that a problem
too large for the array is refused.  It is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_1411_0330_gb300 import lsh  # noqa: E402

EL = np.array([[0.8333333333333334, 0.38461538461538464], [5.555555555555555, 4.166666666666667]])


def rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


def _call_noalloc(lib, phase, mods, physics, green, x, y, ref=None, scale=None, stream=None):
    refa = None if ref is None else np.ascontiguousarray(ref, dtype=np.float64)
    s = lsh._problem_struct(ctypes.c_void_p(phase.data_ptr()), False, tuple(phase.shape), physics, green, lsh.FP64,
                            np.ascontiguousarray(mods, dtype=np.float64), refa,
                            None if scale is None else ctypes.c_void_p(scale.data_ptr()))
    stream = stream if stream is not None else torch.cuda.current_stream()
    return lib.lsh_apply_noalloc(ctypes.byref(s), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                 ctypes.c_void_p(stream.cuda_stream))


SCALAR3 = np.array([np.diag([1.0, 2.0, 3.0]), np.diag([4.0, 2.0, 7.0])])


@pytest.mark.parametrize("shape,physics,green,mods,ref,with_scale", [
    ((16, 20, 24), lsh.ELASTIC, lsh.FILTERED, EL, None, False),
    ((32, 32), lsh.SCALAR, lsh.TRUNCATED, np.array([np.eye(2), 10 * np.eye(2)]), 5.5 * np.eye(2), False),
    ((9, 10, 12), lsh.SCALAR, lsh.FILTERED, SCALAR3, None, False),
    ((10, 12, 8), lsh.SCALAR, lsh.FD, SCALAR3, None, False),
    ((8, 12, 10), lsh.ELASTIC, lsh.TRUNCATED, EL, np.array([0.25, 0.15]), True),
    ((64, 64, 64), lsh.ELASTIC, lsh.FILTERED, EL, None, False),  # the largest cubic elastic grid the array holds
])
def test_noalloc_apply_matches_lsh_apply_twice(shape, physics, green, mods, ref, with_scale):
    """Two calls in a row equal lsh_apply on a handle of the same problem to 1e-12, and the
    oracle's operator (smaller grids) to the same tolerance."""
    lib = lsh.load_library()
    rng = np.random.default_rng(2024)
    ph_np = (rng.random(shape) < 0.4).astype(np.uint8)
    phase = torch.from_numpy(ph_np).cuda()
    sc_np = rng.uniform(0.5, 2.0, shape).astype(np.float32) if with_scale else None
    scale = torch.from_numpy(sc_np).cuda() if with_scale else None
    h = lsh.Handle(phase, mods, physics=physics, green=green, ref=ref, scale=scale)
    P = oracle.Problem(ph_np, mods, physics=physics, green=green, ref=ref,
                       scale=None if sc_np is None else sc_np.astype(np.float64)) if ph_np.size <= 4096 else None
    for call in range(2):  # the shared scratch keeps the previous call's contents
        x = torch.from_numpy(rng.standard_normal(h.field_shape)).cuda()
        y_ref = h.apply(x)
        y = torch.full_like(x, float("nan"))
        assert _call_noalloc(lib, phase, mods, physics, green, x, y, ref, scale) == lsh.OK, call
        torch.cuda.synchronize()
        assert rel(y, y_ref) < 1e-12, (call, rel(y, y_ref))
        if P is not None:
            yo = torch.from_numpy(oracle.apply(P, x.cpu().numpy()))
            assert rel(y.cpu(), yo) < 1e-12, (call, rel(y.cpu(), yo))


def test_noalloc_refuses_a_capturing_stream():
    """A call copies host tables and synchronises its stream, which stream capture
    forbids: it returns LSH_ERR_INVALID_ARG and enqueues nothing."""
    lib = lsh.load_library()
    phase = torch.zeros((8, 8, 8), dtype=torch.uint8, device="cuda")
    phase[2:5, 2:6, 1:7] = 1
    x = torch.ones((6, 8, 8, 8), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        status = _call_noalloc(lib, phase, EL, lsh.ELASTIC, lsh.FILTERED, x, y, stream=side)
    assert status == lsh.ERR_INVALID_ARG
    assert _call_noalloc(lib, phase, EL, lsh.ELASTIC, lsh.FILTERED, x, y) == lsh.OK


def test_noalloc_rejects_problems_beyond_its_scratch():
    lib = lsh.load_library()
    phase = torch.zeros((128, 128, 128), dtype=torch.uint8, device="cuda")
    x = torch.zeros((6, 128, 128, 128), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    assert _call_noalloc(lib, phase, EL, lsh.ELASTIC, lsh.FILTERED, x, y) == lsh.ERR_UNSUPPORTED_SIZE
