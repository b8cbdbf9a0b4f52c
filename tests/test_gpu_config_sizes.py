"""Oracle parity at the sizes of the benchmark configurations, through the C ABI.

* 256^3 (the mixed-precision configuration: the 128^3 packing's sphere centres at
  radius 16 voxels): one operator application of Eq. (13) in FP64, in
  double-float (the arithmetic of the mixed solver's refinement residual) and in
  FP32 with the autotuned kernel variants, element by element against the FP64
  CPU oracle, filtered and truncated Green operators.
* 96^3 and 48^3 (the radix-3 grids of the batched configuration): FP64,
  double-float and FP32 (plane passes) applications against the oracle.

Tolerances (max |difference| / max |oracle|): FP64 1e-12, double-float 1e-13,
FP32 2e-5 -- rounding of FFTs of log2 V <= 24 levels times the local contrast.
"""
import numpy as np
import pytest

from helpers import k_mu

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from paper_1411_0330_gb300 import lsh  # noqa: E402
from paper_1411_0330_gb300 import microstructures as ms  # noqa: E402

KM, MUM = k_mu(1.0, 0.3)
KI, MUI = k_mu(10.0, 0.2)
EL = np.array([[KM, MUM], [KI, MUI]])


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


@pytest.fixture(scope="module")
def spheres256():
    _, cen, r = ms.sphere_microstructure(128, 8.0, 0.3, seed=1411)
    return ms.voxelize_spheres(256, cen, r)


@pytest.mark.parametrize("green", [lsh.FILTERED, lsh.TRUNCATED])
def test_apply_256_fp64_double_float_fp32_match_oracle(spheres256, green):
    ph = spheres256
    rng = np.random.default_rng(256 + green)
    x = rng.standard_normal((6,) + ph.shape)
    yo = oracle.apply(oracle.Problem(ph, EL, physics=1, green=green), x)
    xd = torch.from_numpy(x).cuda()
    ph_d = torch.from_numpy(ph).cuda()
    h64 = lsh.Handle(ph_d, EL, physics=lsh.ELASTIC, green=green, max_systems=1)
    e64 = rel(h64.apply(xd).cpu().numpy(), yo)
    h64.close()
    del h64
    torch.cuda.empty_cache()
    assert e64 < 1e-12, e64
    hmx = lsh.Handle(ph_d, EL, physics=lsh.ELASTIC, green=green, precision=lsh.MIXED, max_systems=1)
    edf = rel(hmx.apply(xd, double_float=True).cpu().numpy(), yo)
    assert edf < 1e-13, edf
    hmx.autotune()
    e32 = rel(hmx.apply(xd.float()).cpu().numpy(), yo)
    assert e32 < 2e-5, e32


@pytest.mark.parametrize("n", [48, 96])
def test_apply_radix3_grids_fp64_and_fp32_match_oracle(n):
    """The batched configuration's radix-3 grids: a seeded packing (r = N/16 voxels,
    f = 0.25); FP64 on the mixed-radix shared-memory passes, FP32 on the plane passes."""
    ph, _, _ = ms.sphere_microstructure(n, n / 16.0, 0.25, seed=1411 + n)
    rng = np.random.default_rng(n)
    x = rng.standard_normal((6,) + ph.shape)
    yo = oracle.apply(oracle.Problem(ph, EL, physics=1, green=1), x)
    ph_d = torch.from_numpy(ph).cuda()
    xd = torch.from_numpy(x).cuda()
    h64 = lsh.Handle(ph_d, EL, physics=lsh.ELASTIC, green=lsh.FILTERED, max_systems=1)
    assert rel(h64.apply(xd).cpu().numpy(), yo) < 1e-12
    hmx = lsh.Handle(ph_d, EL, physics=lsh.ELASTIC, green=lsh.FILTERED, precision=lsh.MIXED, max_systems=1)
    assert hmx.autotune()["y_variant"] == 2
    assert rel(hmx.apply(xd).cpu().numpy(), yo) < 1e-12  # the mixed handle's FP64 operator
    assert rel(hmx.apply(xd, double_float=True).cpu().numpy(), yo) < 1e-13  # the refinement residual's
    assert rel(hmx.apply(xd.float()).cpu().numpy(), yo) < 2e-5
