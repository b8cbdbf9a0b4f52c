"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: the spec bar is a relative error <= 1e-10 on A*/C* for the
FP64 solver and <= 1e-8 for the mixed-precision solver; single operator
applications in FP64 must agree to 1e-12 of the output's max norm (a few
hundred ulps of FFT rounding), FP32 applications to 2e-5.
"""
import numpy as np
import pytest

from helpers import iso_mandel, k_mu

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


def _scalar_mods(d, seed, nphase=3):
    rng = np.random.default_rng(seed)
    return np.array([np.diag(rng.uniform(1.0, 10.0, d)) for _ in range(nphase)])


APPLY_CASES = [
    # (numpy shape (n2, n1, n0) or (n1, n0), physics, green)
    ((32, 32), 0, 0),
    ((12, 10), 0, 1),
    ((9, 15), 0, 0),      # odd lengths, radices 3 and 5
    ((14, 7), 0, 1),      # radix 7
    ((10, 12, 16), 0, 1),
    ((8, 8, 8), 1, 0),
    ((8, 8, 8), 1, 1),
    ((6, 10, 12), 1, 1),  # ragged kx tiles, radix 3 and 5
    ((5, 7, 9), 1, 0),    # all odd
    ((1, 6, 8), 1, 1),    # degenerate axis
    ((24, 20, 18), 1, 1),
]


@pytest.mark.parametrize("shape,physics,green", APPLY_CASES)
def test_apply_matches_oracle(shape, physics, green):
    rng = np.random.default_rng(hash((shape, physics, green)) % 2**32)
    d = len(shape)
    if physics == 1:
        ph = (rng.random(shape) < 0.4).astype(np.uint8)
        mods = EL
    else:
        ph = rng.integers(0, 3, shape).astype(np.uint8)
        mods = _scalar_mods(d, 3)
    P = oracle.Problem(ph, mods, physics=physics, green=green)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=physics, green=green)
    x = rng.standard_normal(P.field_shape)
    y = h.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    yo = oracle.apply(P, x)
    assert rel(y, yo) < 1e-12


def test_apply_with_inactive_voxels_and_reference():
    """Voxels whose phase equals A0 are outside I0: the output vanishes there."""
    ph = np.zeros((12, 16), np.uint8)
    ph[3:9, 4:11] = 1
    mods = np.array([np.eye(2) * 2.0, np.eye(2) * 7.0])
    ref = np.eye(2) * 2.0
    P = oracle.Problem(ph, mods, green=1, ref=ref)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, green=lsh.FILTERED, ref=ref)
    x = np.random.default_rng(1).standard_normal(P.field_shape)
    y = h.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.all(y[:, ph == 0] == 0)
    assert rel(y, oracle.apply(P, x)) < 1e-12


@pytest.mark.parametrize("green", [0, 1])
def test_apply_fp32_mixed_handle(green):
    rng = np.random.default_rng(5)
    ph = (rng.random((16, 12, 20)) < 0.3).astype(np.uint8)
    P = oracle.Problem(ph, EL, physics=1, green=green)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), EL, physics=lsh.ELASTIC, green=green, precision=lsh.MIXED)
    x = rng.standard_normal(P.field_shape)
    y32 = h.apply(torch.from_numpy(x).float().cuda()).cpu().numpy()
    y64 = h.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    yo = oracle.apply(P, x)
    assert rel(y64, yo) < 1e-12
    assert rel(y32, yo) < 2e-5


def test_config1_square_inclusion_indefinite_reference():
    """32 x 32, k = 1 / 10, k0 = (1 + 10)/2 (indefinite operator), truncated Gamma,
    loads e1, e2, rel. residual 1e-10: A* against the oracle's MINRES solution."""
    ph = ms.square_inclusion(32)
    mods = np.array([np.eye(2), 10 * np.eye(2)])
    ref = 5.5 * np.eye(2)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, green=lsh.TRUNCATED, ref=ref)
    Ao, _ = oracle.effective(oracle.Problem(ph, mods, green=0, ref=ref), tol=1e-13)
    # AUTO runs MINRES here (phases on both sides of k0); CG as the configuration states
    for solver in (lsh.SOLVER_AUTO, lsh.SOLVER_CG, lsh.SOLVER_MINRES):
        A, infos = h.effective(tol=1e-10, solver=solver)
        assert rel(A, Ao) < 1e-10, (solver, A, Ao, infos)
        assert abs(A[0, 1]) < 1e-10 and abs(A[0, 0] - A[1, 1]) < 1e-10
        assert all(i["status"] == 0 and i["relres"] <= 1e-10 for i in infos)
    # truncated Gamma: A* does not depend on the reference medium (Table 1)
    h2 = lsh.Handle(torch.from_numpy(ph).cuda(), mods, green=lsh.TRUNCATED, ref=0.5 * np.eye(2))
    A2, _ = h2.effective(tol=1e-12)
    assert rel(A2, Ao) < 1e-9


@pytest.mark.parametrize("precision", [0, 1])
def test_minres_indefinite_elastic_matches_oracle(precision):
    """Elastic spheres with the reference between the phases (mu0 above the matrix,
    below the inclusions): K is indefinite, AUTO solves with MINRES (FP64 also on a
    mixed handle), batched over the 6 loads, warm start included."""
    ph, _, _ = ms.sphere_microstructure(12, 1.5, 0.25, seed=31)
    ref = np.array([2.0 * KM, 2.0 * MUM])  # between the matrix and inclusion moduli
    h = lsh.Handle(torch.from_numpy(ph).cuda(), EL, physics=lsh.ELASTIC, green=lsh.FILTERED, ref=ref,
                   precision=precision)
    A, infos = h.effective(tol=1e-11)
    Ao, _ = oracle.effective(oracle.Problem(ph, EL, physics=1, green=1, ref=ref), tol=1e-13)
    assert rel(A, Ao) < 1e-10, rel(A, Ao)
    assert all(i["status"] == 0 for i in infos)
    load = np.array([0.2, -0.1, 0.4, 0.0, 0.3, 0.1])
    tau, info = h.solve(load, tol=1e-11)
    to, _, _ = oracle.solve(oracle.Problem(ph, EL, physics=1, green=1, ref=ref), load, tol=1e-13)
    assert rel(tau.cpu().numpy(), to) < 1e-9
    tau2, info2 = h.solve(load, tau=tau.clone(), tol=1e-11, warm_start=True)
    assert info2["iters"] <= 2 and rel(tau2.cpu().numpy(), to) < 1e-9


@pytest.mark.parametrize("green", [0, 1])
def test_effective_spheres_fp64(green):
    ph, _, _ = ms.sphere_microstructure(16, 2.0, 0.3, seed=1411)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), EL, physics=lsh.ELASTIC, green=green)
    A, infos = h.effective(tol=1e-12)
    Ao, info_o = oracle.effective(oracle.Problem(ph, EL, physics=1, green=green), tol=1e-12)
    assert rel(A, Ao) < 1e-10
    assert np.allclose(A, A.T, atol=1e-10 * np.abs(A).max())
    for i, inf in enumerate(infos):
        assert inf["status"] == 0 and inf["relres"] <= 1e-12
        # same algorithm, same tolerance: iteration counts agree up to rounding
        assert abs(inf["iters"] - info_o[i, 0]) <= 2


@pytest.mark.parametrize("green", [0, 1])
def test_effective_mixed_precision(green):
    ph, _, _ = ms.sphere_microstructure(16, 2.0, 0.3, seed=1412)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), EL, physics=lsh.ELASTIC, green=green, precision=lsh.MIXED)
    A, infos = h.effective(tol=1e-10)
    Ao, _ = oracle.effective(oracle.Problem(ph, EL, physics=1, green=green), tol=1e-13)
    assert rel(A, Ao) < 1e-8, rel(A, Ao)
    for inf in infos:
        assert inf["status"] == 0 and inf["relres"] <= 1e-10 and inf["outer"] >= 1


def test_high_contrast_mixed():
    ph, _, _ = ms.sphere_microstructure(16, 2.0, 0.3, seed=3)
    mods = np.array([[KM, MUM], list(k_mu(1000.0, 0.2))])
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=lsh.ELASTIC, green=lsh.FILTERED, precision=lsh.MIXED)
    A, infos = h.effective(tol=1e-10, maxit=20000)
    Ao, _ = oracle.effective(oracle.Problem(ph, mods, physics=1, green=1), tol=1e-13, maxit=20000)
    assert rel(A, Ao) < 1e-8, rel(A, Ao)


def test_uniform_medium_and_empty_I0():
    K1, mu1 = k_mu(2.0, 0.25)
    ph = np.zeros((8, 8, 8), np.uint8)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), np.array([[K1, mu1]]), physics=lsh.ELASTIC, green=lsh.FILTERED,
                   ref=np.array([0.4, 0.2]))
    A, infos = h.effective(tol=1e-14)
    assert np.allclose(A, iso_mandel(K1, mu1), atol=1e-13)
    assert all(i["iters"] <= 2 for i in infos)
    # A_phase == A0 everywhere: I0 empty, tau = 0, A* = A0, no iteration
    h0 = lsh.Handle(torch.from_numpy(ph).cuda(), np.array([[K1, mu1]]), physics=lsh.ELASTIC,
                    green=lsh.FILTERED, ref=np.array([K1, mu1]))
    A0, infos0 = h0.effective(tol=1e-10, return_tau=False)
    assert np.allclose(A0, iso_mandel(K1, mu1), atol=1e-14)
    assert all(i["iters"] == 0 for i in infos0)


def test_solve_warm_start_and_determinism():
    ph, _, _ = ms.sphere_microstructure(16, 2.0, 0.25, seed=9)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), EL, physics=lsh.ELASTIC, green=lsh.FILTERED)
    load = np.array([0.0, 0.0, 0.0, 0.0, 0.0, 1.0])
    t1, i1 = h.solve(load, tol=1e-11)
    t2, i2 = h.solve(load, tol=1e-11)
    assert torch.equal(t1, t2) and i1 == i2
    t3, i3 = h.solve(load, tau=t1.clone(), tol=1e-11, warm_start=True)
    assert i3["iters"] <= 1
    to, _, _ = oracle.solve(oracle.Problem(ph, EL, physics=1, green=1), load, tol=1e-13)
    assert rel(t1.cpu().numpy(), to) < 1e-9


def test_set_microstructure_matches_fresh_handle():
    ph1, _, _ = ms.sphere_microstructure(16, 2.0, 0.2, seed=21)
    ph2, _, _ = ms.sphere_microstructure(16, 2.0, 0.3, seed=22)
    h = lsh.Handle(torch.from_numpy(ph1).cuda(), EL, physics=lsh.ELASTIC, green=lsh.TRUNCATED)
    h.set_microstructure(ph2)  # from host memory
    A, _ = h.effective(tol=1e-12)
    Ao, _ = oracle.effective(oracle.Problem(ph2, EL, physics=1, green=0), tol=1e-13)
    assert rel(A, Ao) < 1e-10


def test_scale_gradient_matches_oracle():
    rng = np.random.default_rng(4)
    n = 6
    ph = (rng.random((n, n, n)) < 0.4).astype(np.uint8)
    s = rng.uniform(0.5, 2.0, (n, n, n)).astype(np.float32)
    ref = np.array([0.25 * KM, 0.25 * MUM])
    h = lsh.Handle(torch.from_numpy(ph).cuda(), EL, physics=lsh.ELASTIC, green=lsh.FILTERED, ref=ref,
                   scale=torch.from_numpy(s).cuda())
    A, infos, tau = h.effective(tol=1e-13, return_tau=True)
    W = np.zeros((6, 6)); W[0, 0] = 1.0; W[5, 5] = 0.5
    g = h.effective_grad(tau, W).cpu().numpy()
    P = oracle.Problem(ph, EL, physics=1, green=1, ref=ref, scale=s.astype(np.float64))
    Ao, _, tau_o = oracle.effective(P, tol=1e-13, return_tau=True)
    go = oracle.scale_gradient(P, tau_o, W)
    assert rel(A, Ao) < 1e-10
    assert rel(tau.cpu().numpy(), tau_o) < 1e-9
    assert rel(g, go) < 1e-9


# ------------------------------------------------------------------ full size (128^3, the benchmark's workload)
@pytest.fixture(scope="module")
def spheres128():
    ph, cen, r = ms.sphere_microstructure(128, 8.0, 0.3, seed=1411)
    return ph


@pytest.mark.parametrize("green", [0, 1])
def test_full_size_apply_matches_oracle(spheres128, green):
    ph = spheres128
    rng = np.random.default_rng(128)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), EL, physics=lsh.ELASTIC, green=green)
    x = rng.standard_normal((6,) + ph.shape)
    y = h.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    yo = oracle.apply(oracle.Problem(ph, EL, physics=1, green=green), x)
    assert rel(y, yo) < 1e-12


def test_full_size_solve_properties(spheres128):
    """128^3 FP64, filtered Gamma: the GPU polarisation satisfies the oracle's Eq. (13)
    to the requested tolerance, and C* is symmetric and between C0 and Voigt."""
    ph = spheres128
    h = lsh.Handle(torch.from_numpy(ph).cuda(), EL, physics=lsh.ELASTIC, green=lsh.FILTERED)
    A, infos, tau = h.effective(tol=1e-10, return_tau=True)
    P = oracle.Problem(ph, EL, physics=1, green=1)
    for j in (0, 5):
        t = tau[j].cpu().numpy()
        r = oracle.apply(P, t)
        b = np.zeros_like(t)
        b[j] = 1.0
        assert np.linalg.norm(b - r) / np.linalg.norm(b) < 2e-10
    assert np.allclose(A, A.T, atol=1e-9 * np.abs(A).max())
    C0 = iso_mandel(*P.ref)
    f = ph.mean()
    Cv = (1 - f) * iso_mandel(KM, MUM) + f * iso_mandel(KI, MUI)
    assert np.linalg.eigvalsh(A - C0).min() > 0 and np.linalg.eigvalsh(Cv - A).min() > 0


def test_autograd_effective_tensor_gradient():
    """torch.autograd over the C ABI: d(C*_1111 + C*_1212)/ds against the oracle's gradient
    and central differences of the oracle's dense solves."""
    from paper_1411_0330_gb300.autograd import effective_tensor
    rng = np.random.default_rng(12)
    n = 4
    ph = (rng.random((n, n, n)) < 0.4).astype(np.uint8)
    s0 = rng.uniform(0.5, 2.0, (n, n, n)).astype(np.float32)
    ref = np.array([0.25 * KM, 0.25 * MUM])
    h = lsh.Handle(torch.from_numpy(ph).cuda(), EL, physics=lsh.ELASTIC, green=lsh.FILTERED, ref=ref,
                   scale=torch.from_numpy(s0).cuda())
    s = torch.from_numpy(s0).cuda().requires_grad_(True)
    A = effective_tensor(s, h, tol=1e-13)
    obj = A[0, 0] + 0.5 * A[5, 5]  # C*_1111 + C*_1212 in Mandel components
    obj.backward()
    g = s.grad.double().cpu().numpy()
    P = oracle.Problem(ph, EL, physics=1, green=1, ref=ref, scale=s0.astype(np.float64))
    _, _, tau_o = oracle.effective(P, tol=1e-13, return_tau=True)
    W = np.zeros((6, 6)); W[0, 0] = 1.0; W[5, 5] = 0.5
    go = oracle.scale_gradient(P, tau_o, W)
    # the gradient is returned in the dtype of s (float32): a few float32 ulps
    assert rel(g, go) < 3e-7

    def obj_dense(sc):
        Pp = oracle.Problem(ph, EL, physics=1, green=1, ref=ref, scale=sc)
        C0 = iso_mandel(*ref)
        t0 = oracle.dense_solve(Pp, np.eye(6)[0])
        t5 = oracle.dense_solve(Pp, np.eye(6)[5])
        return C0[0, 0] + t0[0].mean() + 0.5 * (C0[5, 5] + t5[5].mean())

    hstep = 1e-6
    for idx in [(0, 0, 0), (1, 2, 3), (3, 1, 2)]:
        sp = s0.astype(np.float64); sm = sp.copy()
        sp[idx] += hstep
        sm[idx] -= hstep
        fd = (obj_dense(sp) - obj_dense(sm)) / (2 * hstep)
        assert abs(g[idx] - fd) <= 1e-6 * abs(fd) + 1e-10


# ------------------------------------------------------------------ batching (loads x microstructures)
def _batch(n, fracs, seed0):
    return np.stack([ms.sphere_microstructure(n, 2.0, f, seed=seed0 + i)[0] for i, f in enumerate(fracs)])


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_microstructures_match_oracle(precision):
    """Three 16^3 microstructures x 6 loads solved together (18 systems) = the oracle one by one."""
    phs = _batch(16, [0.1, 0.2, 0.3], 50)
    h = lsh.Handle(torch.from_numpy(phs).cuda(), EL, physics=lsh.ELASTIC, green=lsh.FILTERED, precision=precision,
                   batch=True)
    A, infos = h.effective(tol=1e-11)
    assert A.shape == (3, 6, 6) and len(infos) == 18
    for b in range(3):
        Ao, _ = oracle.effective(oracle.Problem(phs[b], EL, physics=1, green=1), tol=1e-13)
        assert rel(A[b], Ao) < (1e-10 if precision == 0 else 1e-8), (b, rel(A[b], Ao))


def test_waves_of_systems_equal_one_wave():
    """max_systems bounds the workspace; solving in waves gives the same C* bit for bit
    for systems that land in identical positions, and to 1e-12 otherwise."""
    phs = _batch(12, [0.2, 0.3], 70)
    h_all = lsh.Handle(torch.from_numpy(phs).cuda(), EL, physics=lsh.ELASTIC, green=lsh.TRUNCATED, batch=True)
    h_w = lsh.Handle(torch.from_numpy(phs).cuda(), EL, physics=lsh.ELASTIC, green=lsh.TRUNCATED, batch=True,
                     max_systems=5)
    A1, _ = h_all.effective(tol=1e-12)
    A2, _ = h_w.effective(tol=1e-12)
    assert rel(A2, A1) < 1e-12


def test_batched_apply_and_solve():
    phs = _batch(8, [0.2, 0.3, 0.15], 90)
    h = lsh.Handle(torch.from_numpy(phs).cuda(), EL, physics=lsh.ELASTIC, green=lsh.FILTERED, batch=True)
    rng = np.random.default_rng(3)
    x = rng.standard_normal((3, 6, 8, 8, 8))
    y = h.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    load = np.array([0.3, -0.1, 0.2, 0.0, 0.5, -0.4])
    tau, infos = h.solve(load, tol=1e-12)
    for b in range(3):
        P = oracle.Problem(phs[b], EL, physics=1, green=1)
        assert rel(y[b], oracle.apply(P, x[b])) < 1e-12
        to, _, _ = oracle.solve(P, load, tol=1e-13)
        assert rel(tau[b].cpu().numpy(), to) < 1e-9
        assert infos[b]["status"] == 0


@pytest.mark.parametrize("shape,green", [((32, 32), 0), ((12, 10), 1), ((10, 12, 16), 0), ((9, 8, 6), 1)])
def test_apply_fp32_scalar(shape, green):
    rng = np.random.default_rng(sum(shape) + green)
    d = len(shape)
    ph = rng.integers(0, 3, shape).astype(np.uint8)
    mods = _scalar_mods(d, 3)
    P = oracle.Problem(ph, mods, physics=0, green=green)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=0, green=green, precision=lsh.MIXED)
    x = rng.standard_normal(P.field_shape)
    y32 = h.apply(torch.from_numpy(x).float().cuda()).cpu().numpy()
    assert rel(y32, oracle.apply(P, x)) < 2e-5


@pytest.mark.parametrize("precision", [0, 1])
def test_cuda_graphs_equal_direct_launches(precision):
    """Replaying the captured graphs of check_every CG iterations gives the same
    results bit for bit as launching the kernels one by one, with and without
    per-pass profiling (every chunk or one in three), and the graphs follow a
    microstructure change."""
    phs = _batch(12, [0.2, 0.3], 80)
    h = lsh.Handle(torch.from_numpy(phs).cuda(), EL, physics=lsh.ELASTIC, green=lsh.FILTERED, precision=precision,
                   batch=True)
    A_d, i_d = h.effective(tol=1e-11, graphs=False)
    n_d = h.profile_read(reset=True)["launches"]
    A_g, i_g = h.effective(tol=1e-11)
    n_g = h.profile_read(reset=True)["launches"]
    assert np.array_equal(A_d, A_g) and i_d == i_g and n_d == n_g
    h.profile_enable(True)
    A_p, i_p = h.effective(tol=1e-11, check_every=4)
    prof = h.profile_read(reset=True)
    h.profile_enable(False)
    assert np.array_equal(A_p, A_g) and i_p == i_g
    assert prof["timed_iters"] > 0 and all(v > 0 for v in prof["pass_ms"].values())
    # events in one chunk of three: the same results, fewer timed iterations
    h.profile_enable(True, every=3)
    A_s, i_s = h.effective(tol=1e-11, check_every=4)
    prof_s = h.profile_read(reset=True)
    h.profile_enable(False)
    assert np.array_equal(A_s, A_g) and i_s == i_g
    assert 0 < prof_s["timed_iters"] < prof["timed_iters"]
    # new microstructures in the same handle: the cached graphs are re-captured
    phs2 = _batch(12, [0.25, 0.1], 81)
    h.set_microstructure(phs2)
    A2, _ = h.effective(tol=1e-11)
    for b in range(2):
        Ao, _ = oracle.effective(oracle.Problem(phs2[b], EL, physics=1, green=1), tol=1e-13)
        assert rel(A2[b], Ao) < (1e-10 if precision == 0 else 1e-8)


def test_grid_batch_uneven_grids_match_oracle():
    """Microstructures of three grid sizes (radix-2 and radix-3 lengths) solved
    together through lsh_effective_batch (one handle and stream per grid) equal
    the oracle one by one, and the order of the inputs is kept."""
    rng = np.random.default_rng(1411)
    sizes = [8, 12, 8, 16, 12]
    phases = []
    for i, n in enumerate(sizes):
        f = float(rng.uniform(0.1, 0.3))
        ph, _, _ = ms.sphere_microstructure(n, n / 8.0, f, seed=1411 + i)
        phases.append(ph)
    gb = lsh.GridBatch(phases, EL, physics=lsh.ELASTIC, green=lsh.FILTERED, precision=lsh.MIXED)
    assert len(gb.handles) == 3
    A, infos = gb.effective(tol=1e-11)
    for i, ph in enumerate(phases):
        Ao, _ = oracle.effective(oracle.Problem(ph, EL, physics=1, green=1), tol=1e-13)
        assert rel(A[i], Ao) < 1e-8, (i, rel(A[i], Ao))
        assert len(infos[i]) == 6 and all(x["status"] == 0 for x in infos[i])
    # the same handles one after the other give the same tensors bit for bit
    for idx, h in zip(gb.order, gb.handles):
        Ah, _ = h.effective(tol=1e-11)
        for k, i in enumerate(idx):
            assert np.array_equal(Ah[k], A[i])
    gb.close()


@pytest.mark.parametrize("shape,physics", [((8, 32, 20), 1), ((6, 16, 48), 1), ((12, 64, 10), 0), ((4, 128, 36), 0),
                                           ((16, 12, 10), 1), ((32, 16, 18), 1), ((16, 16, 16), 0),
                                           ((64, 6, 12), 1)])
def test_fp32_tma_passes_match_register_passes_and_oracle(shape, physics, monkeypatch):
    """The FP32 y and z passes through the Tensor Memory Accelerator (whole-column
    tiles, ragged last tile, padded rows, Gamma between the z transforms) equal the
    register-FFT passes bit for bit (same arithmetic) and the oracle to FP32
    accuracy."""
    rng = np.random.default_rng(sum(shape))
    if physics == 1:
        ph = (rng.random(shape) < 0.35).astype(np.uint8)
        mods = EL
    else:
        ph = rng.integers(0, 3, shape).astype(np.uint8)
        mods = _scalar_mods(3, 4)
    P = oracle.Problem(ph, mods, physics=physics, green=1)
    x = rng.standard_normal(P.field_shape)
    xt = torch.from_numpy(x).float().cuda()
    h_tma = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=physics, green=1, precision=lsh.MIXED)
    monkeypatch.setenv("LSH_NO_TMA", "1")
    h_reg = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=physics, green=1, precision=lsh.MIXED)
    h_reg.set_variants(0, 0, 0, 0)  # separate register y and z passes (square planes default to the plane passes)
    y_reg = h_reg.apply(xt)
    assert rel(y_reg.cpu().numpy(), oracle.apply(P, x)) < 2e-5
    for zv in range(10):
        try:
            h_tma.set_variants(0, 0, 1, zv)
        except lsh.LSHError as e:
            assert e.status == lsh.ERR_UNSUPPORTED
            continue
        y_tma = h_tma.apply(xt)
        assert torch.equal(y_tma, y_reg), zv
    # the register x passes: other rounding order than the staged ones
    for xf, xv in ((1, 0), (0, 1), (1, 1), (1, 2), (1, 3)):
        try:
            h_tma.set_variants(xf, xv, 1, 0)
        except lsh.LSHError as e:
            assert e.status == lsh.ERR_UNSUPPORTED
            continue
        y_x = h_tma.apply(xt)
        assert rel(y_x.cpu().numpy(), oracle.apply(P, x)) < 2e-5, (xf, xv)
    rep = h_tma.autotune()
    assert rep["z_variant"] in range(12) and rep["y_variant"] in (0, 1, 2) and rep["x_variant"] in (0, 1, 2, 3)
    assert rep["xf_variant"] in (0, 1)
    assert rel(h_tma.apply(xt).cpu().numpy(), oracle.apply(P, x)) < 2e-5


@pytest.mark.parametrize("variants", [(0, 0, 0, 0), (1, 1, 1, 0), (1, 1, 1, 4), (0, 1, 0, 1), (1, 2, 1, 0),
                                      (1, 3, 1, 7)])
def test_mixed_solver_with_each_kernel_variant(variants):
    """The mixed-precision solver (FP32 CG on the forced x / y / z kernel variants,
    FP64 refinement) reaches the oracle's C* to the mixed tolerance whichever
    variants run; unavailable ones are refused with LSH_ERR_UNSUPPORTED."""
    ph, _, _ = ms.sphere_microstructure(32, 4.0, 0.25, seed=77)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), EL, physics=lsh.ELASTIC, green=lsh.FILTERED, precision=lsh.MIXED)
    try:
        h.set_variants(*variants)
    except lsh.LSHError as e:
        assert e.status == lsh.ERR_UNSUPPORTED
        pytest.skip("variant not available for this grid")
    A, infos = h.effective(tol=1e-10)
    Ao, _ = oracle.effective(oracle.Problem(ph, EL, physics=1, green=1), tol=1e-13)
    assert rel(A, Ao) < 1e-8, rel(A, Ao)
    assert all(i["status"] == 0 for i in infos)


@pytest.mark.parametrize("shape,physics,green", [((16, 12, 10), 1, 1), ((64, 12, 18), 1, 0), ((128, 8, 30), 1, 1),
                                                 ((16, 20, 14), 0, 1), ((256, 6, 32), 0, 2), ((32, 4, 40), 0, 0),
                                                 ((64, 10, 6), 0, 2)])
def test_persistent_z_pass_matches_register_z_pass(shape, physics, green):
    """The persistent FP32 z pass (tiles walked with the grid's stride, the next
    tile's columns staged by asynchronous copies, Gamma^h rows prefetched to L2)
    equals the one-tile-per-block register pass bit for bit: truncated (on the fly),
    filtered and (conductivity) finite-difference Gamma^h, three microstructures
    (systems) per launch, ragged last tiles."""
    rng = np.random.default_rng(sum(shape) + 7 * green)
    if physics == 1:
        ph = (rng.random((3,) + shape) < 0.35).astype(np.uint8)
        mods = EL
    else:
        ph = rng.integers(0, 3, (3,) + shape).astype(np.uint8)
        mods = _scalar_mods(3, 4)
    Ps = [oracle.Problem(ph[k], mods, physics=physics, green=green) for k in range(3)]
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=physics, green=green, precision=lsh.MIXED, batch=True)
    x = rng.standard_normal((3,) + Ps[0].field_shape)
    xt = torch.from_numpy(x).float().cuda()
    h.set_variants(0, 0, 0, 0)
    y0 = h.apply(xt)
    h.set_variants(0, 0, 0, 7)
    y7 = h.apply(xt)
    assert torch.equal(y7, y0)
    for k in range(3):
        assert rel(y7[k].cpu().numpy(), oracle.apply(Ps[k], x[k])) < 2e-5


@pytest.mark.parametrize("shape,physics,green", [((32, 32, 32), 1, 1), ((16, 64, 32), 1, 0), ((64, 16, 128), 1, 1),
                                                 ((32, 16, 64), 0, 1), ((16, 32, 16), 0, 0), ((16, 16, 256), 1, 0),
                                                 ((48, 48, 48), 1, 1), ((16, 96, 96), 1, 0), ((96, 32, 32), 0, 1)])
def test_double_float_apply_matches_fp64(shape, physics, green):
    """K x in double-float arithmetic (FP64 fields, every pass on the FP32 pipes
    with 48-bit significands) against the native FP64 passes and the oracle: the
    difference stays at the level of 2^-48 times log N, far below what the
    refinement residual must resolve (1e-11 of ||b||)."""
    rng = np.random.default_rng(sum(shape) + 11 * green + physics)
    if physics == 1:
        ph = (rng.random(shape) < 0.35).astype(np.uint8)
        mods = EL
    else:
        ph = rng.integers(0, 3, shape).astype(np.uint8)
        mods = _scalar_mods(3, 4)
    P = oracle.Problem(ph, mods, physics=physics, green=green)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=physics, green=green, precision=lsh.MIXED)
    x = rng.standard_normal(P.field_shape)
    xt = torch.from_numpy(x).cuda()
    y64 = h.apply(xt).cpu().numpy()
    ydf = h.apply(xt, double_float=True).cpu().numpy()
    yo = oracle.apply(P, x)
    assert rel(ydf, y64) < 1e-13, rel(ydf, y64)
    assert rel(ydf, yo) < 1e-13, rel(ydf, yo)


def test_double_float_residual_solve_matches_native_fp64_residual(monkeypatch):
    """The mixed solver with its refinement residual in double-float (the default
    on such grids) and with the native FP64 residual reach the same C* to the
    solve tolerance, and both the oracle's."""
    ph, _, _ = ms.sphere_microstructure(32, 4.0, 0.25, seed=78)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), EL, physics=lsh.ELASTIC, green=lsh.FILTERED, precision=lsh.MIXED)
    A_df, inf_df = h.effective(tol=1e-10)
    monkeypatch.setenv("LSH_NO_DF", "1")
    h64 = lsh.Handle(torch.from_numpy(ph).cuda(), EL, physics=lsh.ELASTIC, green=lsh.FILTERED, precision=lsh.MIXED)
    A_64, inf_64 = h64.effective(tol=1e-10)
    Ao, _ = oracle.effective(oracle.Problem(ph, EL, physics=1, green=1), tol=1e-13)
    assert rel(A_df, A_64) < 1e-9, rel(A_df, A_64)
    assert rel(A_df, Ao) < 1e-8 and rel(A_64, Ao) < 1e-8
    assert all(i["status"] == 0 and i["relres"] <= 1e-10 for i in inf_df)
    assert sum(i["outer"] for i in inf_df) == sum(i["outer"] for i in inf_64)


@pytest.mark.parametrize("shape,physics", [((16, 256, 32), 1), ((256, 16, 16), 1), ((8, 256, 256), 0)])
def test_length_256_passes_fp64_and_fp32(shape, physics):
    """Lines of 256 points (the largest register-FFT length: 16 x 16 split) along each
    axis, FP64 and FP32 (tuned variants), against the oracle."""
    rng = np.random.default_rng(sum(shape) + physics)
    if physics == 1:
        ph = (rng.random(shape) < 0.3).astype(np.uint8)
        mods = EL
    else:
        ph = rng.integers(0, 2, shape).astype(np.uint8)
        mods = _scalar_mods(3, 6, nphase=2)
    P = oracle.Problem(ph, mods, physics=physics, green=1)
    x = rng.standard_normal(P.field_shape)
    yo = oracle.apply(P, x)
    h64 = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=physics, green=1)
    assert rel(h64.apply(torch.from_numpy(x).cuda()).cpu().numpy(), yo) < 1e-12
    h32 = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=physics, green=1, precision=lsh.MIXED, tune=True)
    assert rel(h32.apply(torch.from_numpy(x).float().cuda()).cpu().numpy(), yo) < 2e-5


FD_CASES = [((32, 32), 0), ((12, 10), 0), ((9, 15), 0), ((10, 12, 16), 0), ((16, 16, 16), 1), ((5, 7, 9), 0),
            ((32, 64, 16), 1)]


@pytest.mark.parametrize("shape,mixed", FD_CASES)
def test_fd_green_operator_apply_matches_oracle(shape, mixed):
    """The finite-difference Green operator (Sec. 3.2.3, scalar): Hermitian per
    frequency, applied as a real table between half-angle phase rotations; FP64
    (and FP32 on mixed handles) against the oracle's complex formula."""
    rng = np.random.default_rng(sum(shape) + 7)
    d = len(shape)
    ph = rng.integers(0, 3, shape).astype(np.uint8)
    mods = _scalar_mods(d, 5)
    P = oracle.Problem(ph, mods, physics=0, green=2)
    x = rng.standard_normal(P.field_shape)
    yo = oracle.apply(P, x)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, green=lsh.FD, precision=lsh.MIXED if mixed else lsh.FP64,
                   tune=bool(mixed))
    assert rel(h.apply(torch.from_numpy(x).cuda()).cpu().numpy(), yo) < 1e-12
    if mixed:
        assert rel(h.apply(torch.from_numpy(x).float().cuda()).cpu().numpy(), yo) < 2e-5


def test_fd_green_operator_effective_and_reference_independence():
    """A*_h with the finite-difference operator equals the oracle's (FP64 and mixed)
    and, like the truncated one, does not depend on the reference medium (Table 1)."""
    ph = ms.square_inclusion(32)
    mods = np.array([np.eye(2), 10 * np.eye(2)])
    Ao, _ = oracle.effective(oracle.Problem(ph, mods, green=2), tol=1e-13)
    for prec in (lsh.FP64, lsh.MIXED):
        h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, green=lsh.FD, precision=prec)
        A, infos = h.effective(tol=1e-11)
        assert rel(A, Ao) < (1e-10 if prec == lsh.FP64 else 1e-8), (prec, rel(A, Ao))
    h2 = lsh.Handle(torch.from_numpy(ph).cuda(), mods, green=lsh.FD, ref=0.9 * np.eye(2))
    A2, _ = h2.effective(tol=1e-12)
    assert rel(A2, Ao) < 1e-9


def _rotation(d, seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((d, d)))
    return q


@pytest.mark.parametrize("shape,green,given_ref", [((24, 20), 1, True), ((10, 12, 16), 0, True),
                                                    ((16, 16, 16), 1, False), ((9, 15), 0, False)])
def test_anisotropic_commuting_reference(shape, green, given_ref):
    """Scalar conductivity with anisotropic phase tensors that commute with an
    anisotropic reference (common eigenvectors, Eq. (hyp3)): the library works in
    their eigenbasis; apply and A* equal the oracle's full-tensor computation."""
    d = len(shape)
    Q = _rotation(d, sum(shape))
    rng = np.random.default_rng(len(shape) + green)
    mods = np.array([Q @ np.diag(rng.uniform(1.0, 8.0, d)) @ Q.T for _ in range(3)])
    mods = 0.5 * (mods + mods.transpose(0, 2, 1))
    ref = Q @ np.diag(rng.uniform(0.3, 0.6, d)) @ Q.T if given_ref else None
    if ref is not None:
        ref = 0.5 * (ref + ref.T)
    ph = rng.integers(0, 3, shape).astype(np.uint8)
    P = oracle.Problem(ph, mods, physics=0, green=green, ref=ref)
    x = rng.standard_normal(P.field_shape)
    for prec in (lsh.FP64, lsh.MIXED):
        h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, green=green, ref=ref, precision=prec)
        assert rel(h.apply(torch.from_numpy(x).cuda()).cpu().numpy(), oracle.apply(P, x)) < 1e-12
        A, infos = h.effective(tol=1e-11)
        Ao, _ = oracle.effective(P, tol=1e-13)
        assert rel(A, Ao) < (1e-10 if prec == lsh.FP64 else 1e-8), (prec, rel(A, Ao))
        assert np.allclose(A, A.T, atol=1e-9 * np.abs(A).max())


def test_non_commuting_anisotropy_is_refused():
    d = 2
    Q = _rotation(d, 3)
    mods = np.array([np.diag([1.0, 4.0]), Q @ np.diag([2.0, 5.0]) @ Q.T])
    mods = 0.5 * (mods + mods.transpose(0, 2, 1))
    ph = (np.arange(64).reshape(8, 8) % 2).astype(np.uint8)
    with pytest.raises(lsh.LSHError) as e:
        lsh.Handle(torch.from_numpy(ph).cuda(), mods, green=0, ref=np.eye(2) * 0.4)
    assert e.value.status == lsh.ERR_UNSUPPORTED


@pytest.mark.parametrize("shape", [(9, 15), (5, 7, 9), (3, 5, 6)])
def test_mixed_solve_with_odd_field_lengths(shape):
    """Mixed-precision solves where c V is not a multiple of 4 (FP32 systems do not
    start on 16-byte boundaries): the vector kernels fall back to scalar accesses."""
    rng = np.random.default_rng(sum(shape))
    d = len(shape)
    ph = rng.integers(0, 2, shape).astype(np.uint8)
    mods = _scalar_mods(d, 9, nphase=2)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, green=1, precision=lsh.MIXED)
    A, infos = h.effective(tol=1e-11)
    Ao, _ = oracle.effective(oracle.Problem(ph, mods, physics=0, green=1), tol=1e-13)
    assert rel(A, Ao) < 1e-8 and all(i["status"] == 0 for i in infos)


def test_basic_scheme_matches_oracle():
    """The Moulinec-Suquet fixed point (tau <- tau + (A - A0)(b - K tau)) with the
    reference between the phases converges to the same A* as the oracle; with the
    soft default reference it does not converge and says so."""
    ph = ms.square_inclusion(32)
    mods = np.array([np.eye(2), 10 * np.eye(2)])
    ref = 5.5 * np.eye(2)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, green=lsh.TRUNCATED, ref=ref)
    A, infos = h.effective(tol=1e-10, solver=lsh.SOLVER_BASIC, maxit=2000)
    Ao, _ = oracle.effective(oracle.Problem(ph, mods, green=0, ref=ref), tol=1e-13)
    assert rel(A, Ao) < 1e-9, (A, Ao, infos)
    assert all(i["status"] == 0 and i["relres"] <= 1e-10 for i in infos)
    # elasticity, mixed handle (runs in FP64), reference at the mean of the phases
    phs, _, _ = ms.sphere_microstructure(12, 1.5, 0.2, seed=41)
    refe = 0.5 * (EL[0] + EL[1])
    he = lsh.Handle(torch.from_numpy(phs).cuda(), EL, physics=lsh.ELASTIC, green=lsh.FILTERED, ref=refe,
                    precision=lsh.MIXED)
    Ae, inf_e = he.effective(tol=1e-10, solver=lsh.SOLVER_BASIC, maxit=3000)
    Aeo, _ = oracle.effective(oracle.Problem(phs, EL, physics=1, green=1, ref=refe), tol=1e-13)
    assert rel(Ae, Aeo) < 1e-9, rel(Ae, Aeo)
    # soft reference: the fixed point diverges
    hs = lsh.Handle(torch.from_numpy(ph).cuda(), mods, green=lsh.TRUNCATED)
    _, inf_s = hs.effective(tol=1e-10, solver=lsh.SOLVER_BASIC, maxit=40, raise_on_fail=False)
    assert all(i["status"] != 0 for i in inf_s)


@pytest.mark.parametrize("physics,prec", [(1, lsh.FP64), (1, lsh.MIXED), (0, lsh.FP64), (0, lsh.MIXED)])
def test_subvoxel_averaging_matches_oracle(physics, prec):
    """Voxels with a volume fraction f of phase 1 carry the averaged local operator
    f M1 + (1 - f) M0 of Eq. (def_ah): apply and A* equal the oracle's."""
    n = 12 if physics == 1 else 16
    _, cen, r = ms.sphere_microstructure(n, n / 6.0, 0.25, seed=61)
    f = ms.sphere_fractions(n, cen, r, sub=4)
    if physics == 0:
        f = f[0]  # a 2D slice
        mods = np.array([np.diag([1.0, 1.5]), np.diag([8.0, 6.0])])
    else:
        mods = EL
    ph = np.zeros(f.shape, np.uint8)
    P = oracle.Problem(ph, mods, physics=physics, green=1, frac=f.astype(np.float64))
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, physics=physics, green=1, precision=prec,
                   fraction=torch.from_numpy(f).cuda())
    rng = np.random.default_rng(5)
    x = rng.standard_normal(P.field_shape)
    assert rel(h.apply(torch.from_numpy(x).cuda()).cpu().numpy(), oracle.apply(P, x)) < 1e-12
    A, infos = h.effective(tol=1e-11)
    Ao, _ = oracle.effective(P, tol=1e-13)
    assert rel(A, Ao) < (1e-10 if prec == lsh.FP64 else 1e-8), rel(A, Ao)
    # the fractions are what matters: the phase map is not read
    h.set_microstructure(np.ones(f.shape, np.uint8), f)
    A2, _ = h.effective(tol=1e-11)
    assert rel(A2, Ao) < (1e-10 if prec == lsh.FP64 else 1e-8)


def test_bounded_wait_gives_up_and_the_handle_stays_usable():
    """The give-up path of the bounded barrier waits: a wait on a barrier that never
    completes (two arrivals expected, one given, no copy in flight) runs out after the
    limit, the fault word surfaces as LSH_ERR_CUDA, is cleared, and the handle's next
    operator application is correct."""
    rng = np.random.default_rng(77)
    ph = (rng.random((16, 16, 16)) < 0.3).astype(np.uint8)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), EL, physics=lsh.ELASTIC, green=lsh.FILTERED, precision=lsh.MIXED)
    assert h.check_bounded_wait(0.02) == lsh.ERR_CUDA
    assert h.check_bounded_wait(0.001) == lsh.ERR_CUDA  # the word was cleared and set again
    P = oracle.Problem(ph, EL, physics=1, green=1)
    x = rng.standard_normal(P.field_shape)
    assert rel(h.apply(torch.from_numpy(x).cuda()).cpu().numpy(), oracle.apply(P, x)) < 1e-12
    assert rel(h.apply(torch.from_numpy(x).float().cuda()).cpu().numpy(), oracle.apply(P, x)) < 2e-5
    A, infos = h.effective(tol=1e-10)
    assert all(i["status"] == 0 for i in infos)


def test_symmlq_indefinite_scalar_and_elastic_match_oracle():
    """SYMMLQ (the indefinite-system solver the paper names, Sec. 1) reaches the
    unique solution of Eq. (13): the 2D square inclusion with k0 = (1 + 10) / 2
    (indefinite K) and elastic spheres with the reference between the phases, A*
    against the oracle; its reported residual is the CG point's."""
    ph = ms.square_inclusion(32)
    mods = np.array([np.eye(2), 10 * np.eye(2)])
    ref = 5.5 * np.eye(2)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), mods, green=lsh.TRUNCATED, ref=ref)
    Ao, _ = oracle.effective(oracle.Problem(ph, mods, green=0, ref=ref), tol=1e-13)
    A, infos = h.effective(tol=1e-11, solver=lsh.SOLVER_SYMMLQ)
    assert rel(A, Ao) < 1e-10, rel(A, Ao)
    assert all(i["status"] == 0 and i["relres"] <= 1e-11 for i in infos)
    _, inf_m = h.effective(tol=1e-11, solver=lsh.SOLVER_MINRES)
    # the same Krylov spaces: the CG point needs about as many iterations as MINRES
    assert all(a["iters"] <= 1.5 * b["iters"] + 10 for a, b in zip(infos, inf_m))
    ph3, _, _ = ms.sphere_microstructure(12, 1.5, 0.25, seed=31)
    ref3 = np.array([2.0 * KM, 2.0 * MUM])
    h3 = lsh.Handle(torch.from_numpy(ph3).cuda(), EL, physics=lsh.ELASTIC, green=lsh.FILTERED, ref=ref3)
    P3 = oracle.Problem(ph3, EL, physics=1, green=1, ref=ref3)
    A3, inf3 = h3.effective(tol=1e-11, solver=lsh.SOLVER_SYMMLQ)
    Ao3, _ = oracle.effective(P3, tol=1e-13)
    assert rel(A3, Ao3) < 1e-10, rel(A3, Ao3)
    load = np.array([0.2, -0.1, 0.4, 0.0, 0.3, 0.1])
    tau, info = h3.solve(load, tol=1e-11, solver=lsh.SOLVER_SYMMLQ)
    to, _, _ = oracle.solve(P3, load, tol=1e-13)
    assert rel(tau.cpu().numpy(), to) < 1e-9
    # the true residual of the returned polarisation, by the oracle's operator
    inside = np.ones(ph3.shape, bool)  # every phase differs from the reference here: I0 is the whole cell
    b = inside[None] * load[:, None, None, None]
    r = b - oracle.apply(P3, tau.cpu().numpy())
    assert np.linalg.norm(r) <= 2e-11 * np.linalg.norm(b)
    tau2, info2 = h3.solve(load, tau=tau.clone(), tol=1e-11, warm_start=True, solver=lsh.SOLVER_SYMMLQ)
    assert info2["iters"] <= 2 and rel(tau2.cpu().numpy(), to) < 1e-9


def test_symmlq_definite_equals_cg_solution():
    """On a definite operator SYMMLQ's CG point is the CG iterate: same A* as CG."""
    ph, _, _ = ms.sphere_microstructure(16, 2.0, 0.3, seed=8)
    h = lsh.Handle(torch.from_numpy(ph).cuda(), EL, physics=lsh.ELASTIC, green=lsh.TRUNCATED)
    A_cg, _ = h.effective(tol=1e-12, solver=lsh.SOLVER_CG)
    A_sq, inf = h.effective(tol=1e-12, solver=lsh.SOLVER_SYMMLQ)
    assert rel(A_sq, A_cg) < 1e-10
    assert all(i["status"] == 0 for i in inf)
