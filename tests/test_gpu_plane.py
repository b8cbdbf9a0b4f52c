"""The FP32 plane passes (x and y transforms of a z plane in one kernel, z pass on
the ky-major spectrum, radix-3 register FFTs for 48 and 96) against the FP64 CPU
oracle, through the C ABI.

Tolerances as for the other FP32 paths: one operator application to 2e-5 of the
output's max norm (FP32 FFT rounding, O(eps log2 V) times the local contrast),
C* of the mixed solver to 1e-8 of its largest entry.
"""
import json
import os

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
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _problem(shape, physics, seed):
    rng = np.random.default_rng(seed)
    if physics == 1:
        return (rng.random(shape) < 0.35).astype(np.uint8), EL
    ph = rng.integers(0, 3, shape).astype(np.uint8)
    return ph, np.array([np.diag(rng.uniform(1.0, 10.0, 3)) for _ in range(3)])


PLANE_CASES = [
    # numpy shape (nz, ny, nx): every plane length, z lengths of both FFT families,
    # several kx tiles and the Nyquist column, scalar and elastic, all operators
    ((16, 16, 16), 1, 1),
    ((32, 32, 32), 1, 0),
    ((48, 48, 48), 1, 1),
    ((8 * 2, 96, 96), 1, 1),
    ((96, 48, 48), 0, 1),
    ((64, 64, 64), 0, 0),
    ((32, 128, 128), 1, 1),
    ((256, 32, 32), 1, 0),
    ((48, 16, 16), 0, 2),
    ((16, 96, 96), 0, 2),
    ((64, 16, 16), 1, 1),    # elastic z lengths 64 and 128: the fused z pass on the plans 16 x 4, 32 x 4
    ((128, 16, 16), 1, 0),
]


@pytest.mark.parametrize("shape,physics,green", PLANE_CASES)
def test_plane_apply_matches_oracle(shape, physics, green):
    ph, mods = _problem(shape, physics, sum(shape) + physics + green)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=physics, green=green, precision=lsh.MIXED)
    rep = h.autotune()
    assert rep["y_variant"] in (0, 1, 2)
    h.set_variants(0, 0, 2, 0)  # the plane passes
    P = oracle.Problem(ph, mods, physics=physics, green=green)
    x = np.random.default_rng(1).standard_normal(P.field_shape)
    yo = oracle.apply(P, x)
    for zv in (0, 6, 7, 8, 9, 10, 11):
        if zv == 11 and shape[0] > 128:
            # the fused z pass runs the plan N = R1 x 4 with register DFTs of up to 32 points
            with pytest.raises(lsh.LSHError) as e:
                h.set_variants(0, 0, 2, zv)
            assert e.value.status == lsh.ERR_UNSUPPORTED
            continue
        h.set_variants(0, 0, 2, zv)
        y = h.apply(torch.from_numpy(x).float().cuda()).cpu().numpy()
        assert rel(y, yo) < 2e-5, zv


@pytest.mark.parametrize("shape", [(16, 32, 32), (16, 64, 64), (16, 128, 128)])
def test_plane_passes_agree_with_separate_passes(shape):
    """On power-of-two planes both schedules are available: FP32 results within
    FP32 rounding of each other (different transform algorithms)."""
    ph, mods = _problem(shape, 1, 3)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=lsh.ELASTIC, green=lsh.FILTERED, precision=lsh.MIXED)
    x = torch.from_numpy(np.random.default_rng(2).standard_normal(h.field_shape)).float().cuda()
    h.set_variants(1, 3, 1, 0)
    y_sep = h.apply(x).cpu().numpy()
    h.set_variants(0, 0, 2, 0)
    y_pl = h.apply(x).cpu().numpy()
    assert rel(y_pl, y_sep) < 2e-5


@pytest.mark.parametrize("n,green,nsys,zv", [(32, 1, 6, 10), (16, 0, 6, 10), (32, 1, 2, 10), (48, 1, 3, 10),
                                             (32, 1, 6, 11), (16, 0, 4, 11), (48, 1, 3, 11)])
def test_pipelined_z_pass_mixed_effective_matches_oracle(n, green, nsys, zv):
    """The TMA-fed z passes (variant 10, and 11 with the 4-point DFTs and Gamma^h fused)
    inside the mixed solver: C* against the oracle on a seeded packing, with systems
    converging at different iterations (their tiles are skipped) and waves of fewer
    systems than loads.  48^3: the radix-3 packing whose oracle C* is stored under
    tests/golden/."""
    if n == 48:
        ph, mods, green, Ao = _golden("spheres48_f25_s148_filtered")
    else:
        ph, _, _ = ms.sphere_microstructure(n, n / 8.0, 0.25, seed=300 + n)
        mods = EL
        Ao, _ = oracle.effective(oracle.Problem(ph, EL, physics=1, green=green), tol=1e-13)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=lsh.ELASTIC, green=green, precision=lsh.MIXED,
                   max_systems=nsys)
    h.set_variants(0, 0, 2, zv)
    A, infos = h.effective(tol=1e-10)
    assert rel(A, Ao) < 1e-8, rel(A, Ao)
    assert all(i["status"] == 0 for i in infos)


def test_pipelined_z_pass_needs_the_plane_passes():
    """Variant 10 reads the ky-major spectrum: refused with the separate passes."""
    ph, mods = _problem((16, 32, 32), 1, 5)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=lsh.ELASTIC, green=lsh.FILTERED, precision=lsh.MIXED)
    for zv in (10, 11):
        with pytest.raises(lsh.LSHError) as e:
            h.set_variants(1, 3, 1, zv)
        assert e.value.status == lsh.ERR_UNSUPPORTED
    h.set_variants(0, 0, 2, 10)
    h.set_variants(0, 0, 2, 11)
    h256 = lsh.Handle(torch.zeros((256, 16, 16), dtype=torch.uint8).cuda(), mods, physics=lsh.ELASTIC,
                      green=lsh.FILTERED, precision=lsh.MIXED)
    h256.set_variants(0, 0, 2, 10)
    with pytest.raises(lsh.LSHError) as e:
        h256.set_variants(0, 0, 2, 11)  # z length 256 would need a 64-point register DFT
    assert e.value.status == lsh.ERR_UNSUPPORTED


def test_radix3_grids_refuse_separate_passes():
    """48 and 96 planes run the plane passes only (natural y order in every FP32 pass)."""
    ph, mods = _problem((16, 48, 48), 1, 4)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=lsh.ELASTIC, green=lsh.FILTERED, precision=lsh.MIXED)
    with pytest.raises(lsh.LSHError) as e:
        h.set_variants(1, 3, 0, 0)
    assert e.value.status == lsh.ERR_UNSUPPORTED
    with pytest.raises(lsh.LSHError) as e:
        h.set_variants(0, 0, 2, 1)  # TMA z tiles read the x-major spectrum only
    assert e.value.status == lsh.ERR_UNSUPPORTED
    assert h.autotune()["y_variant"] == 2


def _golden(name):
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_cstar.json")) as fh:
        g = json.load(fh)[name]
    ph, _, _ = ms.sphere_microstructure(g["n"], g["radius"], g["fraction"], seed=g["seed"])
    assert abs(ph.mean() - g["realised_fraction"]) < 1e-12  # the same seeded geometry
    return ph, np.array(g["moduli_K_mu"]), g["green"], np.array(g["cstar_mandel"])


@pytest.mark.parametrize("n,green", [(32, 0), (16, 1)])
def test_plane_mixed_effective_matches_oracle(n, green):
    """The mixed solver (FP32 inner CG on the plane passes, FP64 refinement) reaches
    the oracle's C* to the mixed tolerance on a seeded sphere packing."""
    ph, _, _ = ms.sphere_microstructure(n, n / 8.0, 0.25, seed=100 + n)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), EL, physics=lsh.ELASTIC, green=green, precision=lsh.MIXED)
    h.set_variants(0, 0, 2, 0)
    A, infos = h.effective(tol=1e-10)
    Ao, _ = oracle.effective(oracle.Problem(ph, EL, physics=1, green=green), tol=1e-13)
    assert rel(A, Ao) < 1e-8, rel(A, Ao)
    assert all(i["status"] == 0 for i in infos)


@pytest.mark.parametrize("precision", [lsh.MIXED, lsh.FP64])
def test_radix3_effective_48_matches_stored_oracle(precision):
    """48^3 (a radix-3 grid of the batched configuration): C* of the mixed solver (plane
    passes) and of the FP64 solver against the oracle's, stored by
    tests/golden/make_oracle_cstar.py."""
    ph, mods, green, Ao = _golden("spheres48_f25_s148_filtered")
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=lsh.ELASTIC, green=green, precision=precision)
    A, infos = h.effective(tol=1e-11)
    assert rel(A, Ao) < (1e-8 if precision == lsh.MIXED else 1e-10), rel(A, Ao)
    assert all(i["status"] == 0 for i in infos)


def test_plane_cg_graphs_equal_direct_launches():
    """CUDA-graph replay of the plane-pass CG iterations is bit-identical to launching
    the kernels one by one (the reductions are deterministic)."""
    ph, _, _ = ms.sphere_microstructure(32, 4.0, 0.25, seed=5)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), EL, physics=lsh.ELASTIC, green=lsh.FILTERED, precision=lsh.MIXED)
    h.set_variants(0, 0, 2, 0)
    A1, I1 = h.effective(tol=1e-10, graphs=True)
    A2, I2 = h.effective(tol=1e-10, graphs=False)
    assert np.array_equal(A1, A2)
    assert [i["iters"] for i in I1] == [i["iters"] for i in I2]


@pytest.mark.parametrize("kind", ["scale", "fraction"])
def test_plane_apply_with_voxel_fields(kind):
    """Per-voxel scale s (A = s A_phase) and volume fractions (Eq. (def_ah)) enter the
    local term of the plane inverse pass."""
    rng = np.random.default_rng(9)
    shape = (16, 48, 48)
    ph = (rng.random(shape) < 0.3).astype(np.uint8)
    f = rng.uniform(0.5, 2.0, shape).astype(np.float32) if kind == "scale" else \
        rng.uniform(0.0, 1.0, shape).astype(np.float32)
    ref = np.array([0.25 * KM, 0.25 * MUM])
    if kind == "scale":
        h = lsh.Handle(torch.from_numpy(ph).cuda(), EL, physics=lsh.ELASTIC, green=lsh.FILTERED, ref=ref,
                       precision=lsh.MIXED, scale=torch.from_numpy(f).cuda())
        P = oracle.Problem(ph, EL, physics=1, green=1, ref=ref, scale=f.astype(np.float64))
    else:
        ph0 = np.zeros_like(ph)
        h = lsh.Handle(torch.from_numpy(ph0).cuda(), EL, physics=lsh.ELASTIC, green=lsh.FILTERED, ref=ref,
                       precision=lsh.MIXED, fraction=torch.from_numpy(f).cuda())
        P = oracle.Problem(ph0, EL, physics=1, green=1, ref=ref, frac=f.astype(np.float64))
    h.set_variants(0, 0, 2, 0)
    x = rng.standard_normal(P.field_shape)
    y = h.apply(torch.from_numpy(x).float().cuda()).cpu().numpy()
    assert rel(y, oracle.apply(P, x)) < 2e-5


def test_plane_batched_microstructures_match_oracle():
    """Several microstructures of one 48^3 grid in one batch handle (system-major
    planes, per-system reductions, waves of 5 systems straddling microstructures) give
    each microstructure's stored oracle C*."""
    cases = [_golden(k) for k in ("spheres48_f15_s1_r3_filtered", "spheres48_f30_s2_r3_filtered")]
    stack = np.stack([c[0] for c in cases])
    h = lsh.Handle(torch.from_numpy(stack).cuda(), cases[0][1], physics=lsh.ELASTIC, green=cases[0][2],
                   precision=lsh.MIXED, batch=True, max_systems=5)
    A, infos = h.effective(tol=1e-10)
    for b, c in enumerate(cases):
        assert rel(A[b], c[3]) < 1e-8, (b, rel(A[b], c[3]))


def test_plane_apply_with_unaligned_caller_buffers():
    """The plane passes move fields in 16-byte pieces: a caller's FP32 buffers that
    start 4 bytes off a 16-byte boundary are staged through the handle's own, with
    the result of aligned buffers."""
    ph, mods = _problem((16, 32, 32), 0, 21)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=lsh.SCALAR, green=lsh.FILTERED, precision=lsh.MIXED)
    h.set_variants(0, 0, 2, 0)
    n = int(np.prod(h.field_shape))
    xb = torch.from_numpy(np.random.default_rng(3).standard_normal(n + 1)).float().cuda()
    yb = torch.zeros(n + 1, dtype=torch.float32, device="cuda")
    x_un = xb[1:].view(h.field_shape)
    y_un = yb[1:].view(h.field_shape)
    assert x_un.data_ptr() % 16 != 0
    h.apply(x_un, out=y_un)
    y_al = h.apply(x_un.clone())
    assert torch.equal(y_un, y_al)


def _rotation3(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((3, 3)))
    return q


def test_plane_anisotropic_commuting_phases():
    """Scalar conductivity with anisotropic phase tensors commuting with the reference
    (Eq. (hyp3)): the plane schedule works in their common eigenbasis like the other
    passes; FP32 apply on a radix-3 plane and the mixed C* on a power-of-two plane
    against the oracle's full-tensor computation."""
    Q = _rotation3(5)
    rng = np.random.default_rng(6)
    mods = np.array([Q @ np.diag(rng.uniform(1.0, 8.0, 3)) @ Q.T for _ in range(3)])
    mods = 0.5 * (mods + mods.transpose(0, 2, 1))
    ref = Q @ np.diag([0.4, 0.5, 0.35]) @ Q.T
    ref = 0.5 * (ref + ref.T)
    for shape, check_effective in (((16, 48, 48), False), ((16, 32, 32), True)):
        ph = rng.integers(0, 3, shape).astype(np.uint8)
        P = oracle.Problem(ph, mods, physics=0, green=1, ref=ref)
        h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, green=lsh.FILTERED, ref=ref, precision=lsh.MIXED)
        h.set_variants(0, 0, 2, 0)
        x = rng.standard_normal(P.field_shape)
        assert rel(h.apply(torch.from_numpy(x).float().cuda()).cpu().numpy(), oracle.apply(P, x)) < 2e-5
        if check_effective:
            A, _ = h.effective(tol=1e-11)
            Ao, _ = oracle.effective(P, tol=1e-13)
            assert rel(A, Ao) < 1e-8, rel(A, Ao)


def test_plane_batched_apply_matches_oracle():
    """Two microstructures of one radix-3 plane grid in one batch handle: each system's
    planes find their own phase map (FP32 plane apply against the oracle)."""
    rng = np.random.default_rng(12)
    shape = (16, 48, 48)
    phs = [(rng.random(shape) < f).astype(np.uint8) for f in (0.2, 0.45)]
    h = lsh.Handle(torch.from_numpy(np.stack(phs)).cuda(), EL, physics=lsh.ELASTIC, green=lsh.FILTERED,
                   precision=lsh.MIXED, batch=True)
    h.set_variants(0, 0, 2, 0)
    x = rng.standard_normal((2, 6) + shape)
    y = h.apply(torch.from_numpy(x).float().cuda()).cpu().numpy()
    for b, ph in enumerate(phs):
        yo = oracle.apply(oracle.Problem(ph, EL, physics=1, green=1), x[b])
        assert rel(y[b], yo) < 2e-5, b
