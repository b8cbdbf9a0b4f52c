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

from paper_1411_0330_gb300 import lsh  # noqa: E402

EL = np.array([[0.8333333333333334, 0.38461538461538464], [5.555555555555555, 4.166666666666667]])


def rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


def _call_noalloc(lib, phase, mods, physics, green, x, y, ref=None):
    refa = None if ref is None else np.ascontiguousarray(ref, dtype=np.float64)
    s = lsh._problem_struct(ctypes.c_void_p(phase.data_ptr()), False, tuple(phase.shape), physics, green, lsh.FP64,
                            np.ascontiguousarray(mods, dtype=np.float64), refa, None)
    stream = torch.cuda.current_stream()
    return lib.lsh_apply_noalloc(ctypes.byref(s), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                 ctypes.c_void_p(stream.cuda_stream))


@pytest.mark.parametrize("shape,physics,green,mods,ref", [
    ((16, 20, 24), lsh.ELASTIC, lsh.FILTERED, EL, None),
    ((32, 32), lsh.SCALAR, lsh.TRUNCATED, np.array([np.eye(2), 10 * np.eye(2)]), 5.5 * np.eye(2)),
    ((9, 10, 12), lsh.SCALAR, lsh.FILTERED, np.array([np.diag([1.0, 2.0, 3.0]), np.diag([4.0, 2.0, 7.0])]), None),
])
def test_noalloc_apply_matches_lsh_apply_twice(shape, physics, green, mods, ref):
    lib = lsh.load_library()
    rng = np.random.default_rng(2024)
    phase = torch.from_numpy((rng.random(shape) < 0.4).astype(np.uint8)).cuda()
    h = lsh.Handle(phase, mods, physics=physics, green=green, ref=ref)
    for call in range(2):  # the shared scratch keeps the previous call's contents
        x = torch.from_numpy(rng.standard_normal(h.field_shape)).cuda()
        y_ref = h.apply(x)
        y = torch.full_like(x, float("nan"))
        assert _call_noalloc(lib, phase, mods, physics, green, x, y, ref) == lsh.OK, call
        torch.cuda.synchronize()
        assert rel(y, y_ref) < 1e-12, (call, rel(y, y_ref))


def test_noalloc_rejects_problems_beyond_its_scratch():
    lib = lsh.load_library()
    phase = torch.zeros((128, 128, 128), dtype=torch.uint8, device="cuda")
    x = torch.zeros((6, 128, 128, 128), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    assert _call_noalloc(lib, phase, EL, lsh.ELASTIC, lsh.FILTERED, x, y) == lsh.ERR_UNSUPPORTED_SIZE
