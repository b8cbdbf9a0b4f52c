"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Every check compares the oracle with something other than itself: numpy's
FFT, algebraic properties of the Green operators (projector, range, kernel,
trace), closed-form homogenised tensors (uniform media, laminates), an
independent dense direct solve of Eq. (12), bounds, and a finite-difference
derivative.  A plausible slip anywhere (sign, 1/N^d, transposed operand,
dropped filter term, wrong Nyquist rule) fails at least one of them.
"""
import os

import numpy as np
import pytest

from helpers import (hs_bounds_2d, hs_bounds_elastic, iso_mandel, iso_projection, k_mu,
                     laminate_elastic, mandel_to_tensor2, tensor2_to_mandel)
from paper_1411_0330_gb300 import microstructures as ms

RNG = np.random.default_rng(20141102)


# --------------------------------------------------------------------------- DFT (Sec. 3.1)
@pytest.mark.parametrize("shape", [(8, 8), (6, 5), (4, 6, 8), (3, 5, 7), (1, 4, 3), (16, 2)])
def test_dft_matches_numpy(oracle_mod, shape):
    a = RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)
    f = oracle_mod.dft(a, -1)
    assert np.allclose(f, np.fft.fftn(a), atol=1e-12 * np.abs(a).sum())
    b = oracle_mod.dft(a, +1)
    assert np.allclose(b, np.fft.ifftn(a) * a.size, atol=1e-12 * np.abs(a).sum())


@pytest.mark.parametrize("shape", [(4, 4), (3, 5), (2, 3, 4)])
def test_dft_naive_matches_numpy(oracle_mod, shape):
    a = RNG.standard_normal(shape) + 1j * RNG.standard_normal(shape)
    assert np.allclose(oracle_mod.dft(a, -1, naive=True), np.fft.fftn(a), atol=1e-12 * a.size)


# --------------------------------------------------------------------------- Green operators
def _scalar_problem(dim, n, green, A0=None):
    ph = np.zeros((n,) * dim, dtype=np.uint8)
    mods = np.array([np.eye(dim) * 2.0])
    if A0 is None:
        A0 = np.diag(np.arange(1, dim + 1) * 0.7)
    return oracle_mod_problem(ph, mods, 0, green, A0)


def oracle_mod_problem(ph, mods, physics, green, ref):
    import oracle
    return oracle.Problem(ph, mods, physics=physics, green=green, ref=ref)


def _elastic_problem(n, green, K0=1.3, mu0=0.45):
    ph = np.zeros((n, n, n), dtype=np.uint8)
    return oracle_mod_problem(ph, np.array([[3.0, 1.0]]), 1, green, np.array([K0, mu0]))


def test_gamma0_scalar_projector(oracle_mod):
    """Gamma0 A0 Gamma0 = Gamma0, Gamma0 A0 xi = xi, Gamma0 v = 0 for v . xi = 0 (Sec. 2.2.1)."""
    A0 = np.array([[2.0, 0.3, 0.1], [0.3, 1.5, -0.2], [0.1, -0.2, 1.1]])
    P = oracle_mod.Problem(np.zeros((4, 4, 4), np.uint8), np.array([np.eye(3) * 3]), green=0, ref=A0)
    for _ in range(5):
        xi = RNG.standard_normal(3)
        G = oracle_mod.gamma0(P, xi)
        assert np.allclose(G @ A0 @ G, G, atol=1e-14)
        assert np.allclose(G @ A0 @ xi, xi, atol=1e-14)
        v = np.cross(xi, RNG.standard_normal(3))
        assert np.allclose(G @ v, 0, atol=1e-14)
        assert np.allclose(G, G.T)


def test_gamma0_elastic_characterisation(oracle_mod):
    """Gamma0 C0 eps = eps for compatible eps = sym(a x n); Gamma0 tau = 0 when tau n = 0;
    Gamma0 C0 Gamma0 = Gamma0.  These fix the 6x6 operator uniquely."""
    K0, mu0 = 1.3, 0.45
    C0 = iso_mandel(K0, mu0)
    P = _elastic_problem(4, 0, K0, mu0)
    for _ in range(5):
        n = RNG.standard_normal(3)
        G = oracle_mod.gamma0(P, n * 3.7)
        n = n / np.linalg.norm(n)
        a = RNG.standard_normal(3)
        eps = tensor2_to_mandel(0.5 * (np.outer(a, n) + np.outer(n, a)))
        assert np.allclose(G @ C0 @ eps, eps, atol=1e-13)
        # polarisation with zero traction on planes normal to n
        b1 = np.cross(n, RNG.standard_normal(3)); b1 /= np.linalg.norm(b1)
        b2 = np.cross(n, b1)
        tau = tensor2_to_mandel(1.3 * np.outer(b1, b1) - 0.4 * (np.outer(b1, b2) + np.outer(b2, b1)))
        assert np.allclose(mandel_to_tensor2(tau) @ n, 0, atol=1e-14)
        assert np.allclose(G @ tau, 0, atol=1e-13)
        assert np.allclose(G @ C0 @ G, G, atol=1e-13)
        assert np.allclose(G, G.T, atol=1e-15)


@pytest.mark.parametrize("green", [0, 1, 2])
@pytest.mark.parametrize("n", [6, 7])
def test_gamma_hat_scalar_properties(oracle_mod, green, n):
    """Gamma^h_0 = 0; Gamma^h_{N-k} = conj(Gamma^h_k); tr(A0 Gamma^h_k) = 1 for k != 0
    (each term is a rank-one A0-projector and the weights sum to one)."""
    A0 = np.diag([0.7, 1.4, 2.1])
    P = oracle_mod.Problem(np.zeros((n, n, n), np.uint8), np.array([np.eye(3) * 3]), green=green, ref=A0)
    assert np.allclose(oracle_mod.gamma_hat(P, (0, 0, 0)), 0)
    for _ in range(10):
        k = RNG.integers(0, n, 3)
        if not k.any():
            continue
        G = oracle_mod.gamma_hat(P, k)
        Gm = oracle_mod.gamma_hat(P, (-k) % n)
        assert np.allclose(Gm, np.conj(G), atol=1e-14)
        assert np.allclose(G, np.conj(G.T), atol=1e-14)
        nyq = green == 0 and n % 2 == 0 and (k == n // 2).any()
        assert np.isclose(np.trace(A0 @ G).real, 3.0 if nyq else 1.0, atol=1e-13)
        assert np.min(np.linalg.eigvalsh(G)) > -1e-14
        if green != 2:
            assert np.allclose(G.imag, 0)


@pytest.mark.parametrize("green", [0, 1, 2])
def test_gamma_hat_axis_frequencies_equal_gamma0(oracle_mod, green):
    """For k along one axis (and below Nyquist) every discrete operator of Sec. 3.2
    reduces to Gamma0(e_i): filter weights cos^2 + sin^2 = 1 and Gamma0(-e) = Gamma0(e)."""
    A0 = np.diag([0.7, 1.4, 2.1])
    n = 8
    P = oracle_mod.Problem(np.zeros((n, n, n), np.uint8), np.array([np.eye(3) * 3]), green=green, ref=A0)
    for ax in range(3):
        for kk in (1, 2, 3):
            k = [0, 0, 0]
            k[ax] = kk
            G = oracle_mod.gamma_hat(P, k)
            e = np.zeros(3); e[ax] = 1
            assert np.allclose(G, np.outer(e, e) / A0[ax, ax], atol=1e-14)


def test_gamma_hat_truncated_nyquist_rule(oracle_mod):
    """Sec. 3.2.1: for even N and some k_i = N/2 the truncated operator is A0^{-1};
    for odd N there is no such frequency."""
    A0 = np.diag([0.7, 1.4, 2.1])
    P = oracle_mod.Problem(np.zeros((6, 6, 6), np.uint8), np.array([np.eye(3) * 3]), green=0, ref=A0)
    assert np.allclose(oracle_mod.gamma_hat(P, (3, 1, 0)), np.linalg.inv(A0))
    assert np.allclose(oracle_mod.gamma_hat(P, (0, 0, 3)), np.linalg.inv(A0))
    P7 = P.with_(phase=np.zeros((7, 7, 7), np.uint8))
    G = oracle_mod.gamma_hat(P7, (3, 1, 0))
    assert np.isclose(np.trace(A0 @ G).real, 1.0)
    assert np.linalg.matrix_rank(G.real, tol=1e-12) == 1


@pytest.mark.parametrize("green", [0, 1])
def test_gamma_hat_elastic_trace(oracle_mod, green):
    """tr(C0 Gamma^h_k) = 3: each term is a rank-3 C0-projector, weights sum to one;
    at an elastic Nyquist frequency (truncated) Gamma = C0^{-1} so the trace is 6."""
    K0, mu0 = 1.3, 0.45
    C0 = iso_mandel(K0, mu0)
    P = _elastic_problem(6, green, K0, mu0)
    for _ in range(8):
        k = RNG.integers(0, 6, 3)
        if not k.any():
            continue
        G = oracle_mod.gamma_hat(P, k).real
        expect = 6.0 if (green == 0 and (k == 3).any()) else 3.0
        assert np.isclose(np.trace(C0 @ G), expect, atol=1e-12)
        assert np.min(np.linalg.eigvalsh(G)) > -1e-14


# --------------------------------------------------------------------------- the operator of Eq. (13)
def _random_scalar(dim, n, green, seed, nphase=3, sign=+1):
    rng = np.random.default_rng(seed)
    ph = rng.integers(0, nphase, (n,) * dim).astype(np.uint8)
    mods = []
    for i in range(nphase):
        B = rng.standard_normal((dim, dim))
        mods.append(B @ B.T + (2.0 + i) * np.eye(dim))
    mods = np.array(mods)
    ref = np.eye(dim) * (0.5 if sign > 0 else 20.0)
    import oracle
    return oracle.Problem(ph, mods, physics=0, green=green, ref=ref)


def _random_elastic(n, green, seed, contrast=10.0):
    import oracle
    rng = np.random.default_rng(seed)
    ph = (rng.random((n, n, n)) < 0.35).astype(np.uint8)
    Km, mum = k_mu(1.0, 0.3)
    Ki, mui = k_mu(contrast, 0.2)
    return oracle.Problem(ph, np.array([[Km, mum], [Ki, mui]]), physics=1, green=green)


@pytest.mark.parametrize("green", [0, 1, 2])
@pytest.mark.parametrize("dim,n", [(2, 8), (2, 7), (3, 4), (3, 5)])
def test_operator_symmetric(oracle_mod, green, dim, n):
    P = _random_scalar(dim, n, green, seed=dim * 10 + n)
    x = RNG.standard_normal(P.field_shape)
    y = RNG.standard_normal(P.field_shape)
    Kx, Ky = oracle_mod.apply(P, x), oracle_mod.apply(P, y)
    assert np.isclose(np.vdot(Kx, y), np.vdot(x, Ky), rtol=1e-12)


@pytest.mark.parametrize("green", [0, 1])
def test_operator_symmetric_elastic(oracle_mod, green):
    P = _random_elastic(4, green, 3)
    x = RNG.standard_normal(P.field_shape)
    y = RNG.standard_normal(P.field_shape)
    assert np.isclose(np.vdot(oracle_mod.apply(P, x), y), np.vdot(x, oracle_mod.apply(P, y)), rtol=1e-12)


def test_operator_masks_outside_I0(oracle_mod):
    """Voxels with A_beta = A0 are outside I0: the operator ignores and zeroes them (Eq. (4))."""
    ph = np.zeros((6, 6), np.uint8)
    ph[1:4, 2:5] = 1
    P = oracle_mod.Problem(ph, np.array([np.eye(2) * 1.0, np.eye(2) * 4.0]), green=1, ref=np.eye(2) * 1.0)
    x = RNG.standard_normal(P.field_shape)
    y = oracle_mod.apply(P, x)
    assert np.all(y[:, ph == 0] == 0)
    x2 = x.copy()
    x2[:, ph == 0] = 123.0
    assert np.array_equal(oracle_mod.apply(P, x2), y)


# --------------------------------------------------------------------------- solutions
@pytest.mark.parametrize("green", [0, 1, 2])
@pytest.mark.parametrize("dim,n", [(2, 6), (2, 5), (3, 3), (3, 4)])
def test_cg_matches_dense_eq12(oracle_mod, green, dim, n):
    """Matrix-free CG on Eq. (13) equals an LU solve of Eq. (12) assembled by direct sums."""
    P = _random_scalar(dim, n, green, seed=100 + dim * 10 + n)
    load = RNG.standard_normal(dim)
    tau, it, rr = oracle_mod.solve(P, load, tol=1e-14, solver=1)
    dense = oracle_mod.dense_solve(P, load)
    assert np.allclose(tau, dense, rtol=0, atol=1e-11 * np.abs(dense).max())


@pytest.mark.parametrize("green", [0, 1])
def test_elastic_cg_matches_dense(oracle_mod, green):
    P = _random_elastic(4, green, 7)
    load = RNG.standard_normal(6)
    tau, it, rr = oracle_mod.solve(P, load, tol=1e-14, solver=1)
    dense = oracle_mod.dense_solve(P, load)
    assert np.allclose(tau, dense, rtol=0, atol=1e-11 * np.abs(dense).max())


def test_minres_matches_cg_and_dense(oracle_mod):
    P = _random_scalar(2, 8, 1, seed=5)
    load = np.array([0.3, -1.2])
    t_cg, _, _ = oracle_mod.solve(P, load, tol=1e-14, solver=1)
    t_mr, _, _ = oracle_mod.solve(P, load, tol=1e-14, solver=2)
    assert np.allclose(t_cg, t_mr, atol=1e-11)
    # indefinite: reference between the phases -> MINRES vs dense
    ph = ms.square_inclusion(8)
    Pi = oracle_mod.Problem(ph, np.array([np.eye(2), 10 * np.eye(2)]), green=0, ref=5.5 * np.eye(2))
    t_mr, _, _ = oracle_mod.solve(Pi, load, tol=1e-14, solver=2)
    assert np.allclose(t_mr, oracle_mod.dense_solve(Pi, load), atol=1e-11)


@pytest.mark.parametrize("green", [0, 1, 2])
def test_uniform_medium_scalar(oracle_mod, green):
    """A = A1 everywhere: tau = (A1 - A0) p exactly and A* = A1 (Eqs. (3)-(4), (tau_Astar))."""
    A1 = np.array([[3.0, 0.4], [0.4, 2.0]])
    A0 = np.diag([1.0, 0.5])
    P = oracle_mod.Problem(np.zeros((6, 6), np.uint8), A1[None], green=green, ref=A0)
    load = np.array([0.7, -0.2])
    tau, it, _ = oracle_mod.solve(P, load, tol=1e-14)
    # constant fields: K = M there, whose 2 distinct eigenvalues bound the CG iterations
    assert it <= 2
    assert np.allclose(tau.reshape(2, -1).T, (A1 - A0) @ load, atol=1e-14)
    A, _ = oracle_mod.effective(P, tol=1e-14)
    assert np.allclose(A, A1, atol=1e-14)


@pytest.mark.parametrize("green", [0, 1])
def test_uniform_medium_elastic(oracle_mod, green):
    K1, mu1 = k_mu(2.0, 0.25)
    P = oracle_mod.Problem(np.zeros((4, 4, 4), np.uint8), np.array([[K1, mu1]]), physics=1, green=green,
                           ref=np.array([0.4, 0.2]))
    A, info = oracle_mod.effective(P, tol=1e-14)
    assert np.allclose(A, iso_mandel(K1, mu1), atol=1e-13)
    # isotropic M has two distinct eigenvalues (bulk, shear): at most 2 CG iterations
    assert np.all(info[:, 0] <= 2)


def test_reference_equal_to_medium_gives_zero(oracle_mod):
    """A1 = A0: Q0 is empty, tau = 0 and A* = A0 with zero iterations."""
    P = oracle_mod.Problem(np.zeros((5, 5), np.uint8), np.array([np.eye(2) * 2]), green=1, ref=np.eye(2) * 2)
    tau, it, rr = oracle_mod.solve(P, [1.0, 0.0])
    assert it == 0 and np.all(tau == 0)
    A, _ = oracle_mod.effective(P)
    assert np.allclose(A, 2 * np.eye(2))


@pytest.mark.parametrize("green,n,widths", [(0, 8, [(0, 2), (1, 4), (0, 2)]), (1, 9, [(0, 3), (1, 5), (0, 1)]),
                                            (2, 7, [(0, 2), (1, 5)]), (0, 9, [(0, 3), (1, 6)])])
def test_laminate_scalar(oracle_mod, green, n, widths):
    """Layers normal to axis 0: A*_00 = harmonic mean, A*_11 = arithmetic mean (exact for
    the discrete problem: the solution varies along one axis only)."""
    ph = ms.laminate((n, n), 0, widths)
    a = np.array([1.0, 7.0])
    P = oracle_mod.Problem(ph, np.array([a[0] * np.eye(2), a[1] * np.eye(2)]), green=green, ref=0.5 * np.eye(2))
    A, _ = oracle_mod.effective(P, tol=1e-14)
    f1 = ph[0].mean()
    harm = 1.0 / ((1 - f1) / a[0] + f1 / a[1])
    arit = (1 - f1) * a[0] + f1 * a[1]
    assert np.isclose(A[0, 0], harm, rtol=1e-12)
    assert np.isclose(A[1, 1], arit, rtol=1e-12)
    assert abs(A[0, 1]) < 1e-13


@pytest.mark.parametrize("green", [0, 1])
def test_laminate_elastic(oracle_mod, green):
    """Elastic laminate: classical closed form from continuity of in-plane strain and traction."""
    n = 6
    ph = ms.laminate((n, n, n), 1, [(0, 2), (1, 4)])  # normal along axis 1
    K1, mu1 = k_mu(1.0, 0.3)
    K2, mu2 = k_mu(10.0, 0.2)
    P = oracle_mod.Problem(ph, np.array([[K1, mu1], [K2, mu2]]), physics=1, green=green)
    A, _ = oracle_mod.effective(P, tol=1e-14)
    f2 = (ph == 1).mean()
    Ceff = laminate_elastic([iso_mandel(K1, mu1), iso_mandel(K2, mu2)], [1 - f2, f2], axis=1)
    assert np.allclose(A, Ceff, rtol=0, atol=1e-11 * np.abs(Ceff).max())


def test_truncated_independent_of_reference(oracle_mod):
    """Table 1: with the truncated operator A*_h does not depend on A0 (indefinite k0 = 5.5 included)."""
    ph = ms.square_inclusion(16)
    mods = np.array([np.eye(2), 10 * np.eye(2)])
    As = [oracle_mod.effective(oracle_mod.Problem(ph, mods, green=0, ref=k0 * np.eye(2)), tol=1e-13)[0]
          for k0 in (0.5, 5.5, 20.0)]
    assert np.allclose(As[0], As[1], atol=1e-11) and np.allclose(As[0], As[2], atol=1e-11)
    # the filtered operator does depend on A0 (Table 1), so this is a real test
    Af = [oracle_mod.effective(oracle_mod.Problem(ph, mods, green=1, ref=k0 * np.eye(2)), tol=1e-13)[0]
          for k0 in (0.5, 20.0)]
    assert abs(Af[0][0, 0] - Af[1][0, 0]) > 1e-4


def test_config1_square_inclusion(oracle_mod):
    """32x32, square of side 1/2, k = 1 / 10, k0 = 5.5, truncated: symmetric, square
    symmetry, Voigt/reference bounds, and inside the Hashin-Shtrikman bounds."""
    ph = ms.square_inclusion(32)
    P = oracle_mod.Problem(ph, np.array([np.eye(2), 10 * np.eye(2)]), green=0, ref=5.5 * np.eye(2))
    A, info = oracle_mod.effective(P, tol=1e-12)
    assert np.all(info[:, 1] <= 1e-12)
    assert abs(A[0, 1]) < 1e-12 and abs(A[1, 0]) < 1e-12
    assert np.isclose(A[0, 0], A[1, 1], rtol=1e-12)
    lo, hi = hs_bounds_2d(1.0, 10.0, 0.25)
    assert lo <= A[0, 0] <= hi
    assert A[0, 0] <= 0.75 * 1 + 0.25 * 10


@pytest.mark.parametrize("green", [0, 1])
def test_elastic_bounds_and_symmetry(oracle_mod, green):
    """A0 <= C*_h <= <C> (Voigt) when C0 is softer than every phase; C*_h symmetric."""
    P = _random_elastic(6, green, 11)
    A, _ = oracle_mod.effective(P, tol=1e-13)
    assert np.allclose(A, A.T, atol=1e-12)
    C0 = iso_mandel(*P.ref)
    Cs = [iso_mandel(*P.phase_moduli[i]) for i in range(2)]
    f = (P.phase == 1).mean()
    Cv = (1 - f) * Cs[0] + f * Cs[1]
    assert np.min(np.linalg.eigvalsh(A - C0)) > 0
    assert np.min(np.linalg.eigvalsh(Cv - A)) > 0


def test_spheres_inside_hs_bounds(oracle_mod):
    """Isotropic part of C*_h for a 16^3 sphere packing lies near the Hashin-Shtrikman bounds
    (sanity: the discrete value carries an O(h) error, so only a loose bracket)."""
    ph, _, _ = ms.sphere_microstructure(16, 2.0, 0.2, seed=3)
    K1, mu1 = k_mu(1.0, 0.3)
    K2, mu2 = k_mu(10.0, 0.2)
    P = oracle_mod.Problem(ph, np.array([[K1, mu1], [K2, mu2]]), physics=1, green=1)
    A, _ = oracle_mod.effective(P, tol=1e-10)
    K, mu = iso_projection(A)
    f = (ph == 1).mean()
    (Klo, Khi), (mlo, mhi) = hs_bounds_elastic(K1, mu1, K2, mu2, f)
    assert 0.9 * Klo <= K <= Khi and 0.9 * mlo <= mu <= mhi


def test_variational_estimate_matches(oracle_mod):
    P = _random_elastic(4, 1, 21)
    A, _, tau = oracle_mod.effective(P, tol=1e-14, return_tau=True)
    Av = oracle_mod.effective_variational(P, tau)
    assert np.allclose(A, Av, atol=1e-12)


def test_scale_gradient_matches_finite_differences(oracle_mod):
    """d(sum W_ij e_i.C*e_j)/ds_beta = h^d sum W_ij eps_i . C_phase eps_j (derived from the
    symmetric system of Eq. (13)), against central differences of dense solves."""
    rng = np.random.default_rng(4)
    n = 3
    ph = (rng.random((n, n, n)) < 0.4).astype(np.uint8)
    s = rng.uniform(0.5, 2.0, (n, n, n))
    K1, mu1 = k_mu(1.0, 0.3)
    K2, mu2 = k_mu(10.0, 0.2)
    mods = np.array([[K1, mu1], [K2, mu2]])
    ref = np.array([0.25 * K1, 0.25 * mu1])
    W = np.zeros((6, 6)); W[0, 0] = 1.0; W[5, 5] = 0.5

    def objective(sc):
        P = oracle_mod.Problem(ph, mods, physics=1, green=1, ref=ref, scale=sc)
        cols = [oracle_mod.dense_solve(P, np.eye(6)[j]) for j in (0, 5)]
        C00 = P.ref[0] * 0 + iso_mandel(*ref)[0, 0] + cols[0][0].mean()
        C55 = iso_mandel(*ref)[5, 5] + cols[1][5].mean()
        return C00 + 0.5 * C55, cols

    obj, cols = objective(s)
    P = oracle_mod.Problem(ph, mods, physics=1, green=1, ref=ref, scale=s)
    tau_all = np.zeros((6,) + P.field_shape)
    tau_all[0], tau_all[5] = cols
    g = oracle_mod.scale_gradient(P, tau_all, W)
    h = 1e-5
    for idx in [(0, 0, 0), (1, 2, 0), (2, 1, 1)]:
        sp, sm = s.copy(), s.copy()
        sp[idx] += h
        sm[idx] -= h
        fd = (objective(sp)[0] - objective(sm)[0]) / (2 * h)
        assert np.isclose(g[idx], fd, rtol=1e-6, atol=1e-12)


def test_default_reference_rule(oracle_mod):
    K1, mu1 = k_mu(1.0, 0.3)
    K2, mu2 = k_mu(10.0, 0.2)
    ref = oracle_mod.default_reference(3, 1, np.array([[K1, mu1], [K2, mu2]]))
    assert np.isclose(ref[1], mu1 / 2)
    nu0 = (3 * ref[0] - 2 * ref[1]) / (2 * (3 * ref[0] + ref[1]))
    assert np.isclose(nu0, 0.3)


# ---------------------------------------------------------------- sub-voxel averaging, Eq. (def_ah)
def test_fraction_zero_one_reduces_to_phases(oracle_mod):
    """Volume fractions of exactly 0 or 1 give the one-material-per-voxel operator."""
    rng = np.random.default_rng(71)
    ph = (rng.random((6, 7, 8)) < 0.4).astype(np.uint8)
    mods = np.array([k_mu(1.0, 0.3), k_mu(10.0, 0.2)])
    P = oracle_mod.Problem(ph, mods, physics=oracle_mod.ELASTIC, green=oracle_mod.FILTERED)
    Pf = P.with_(frac=ph.astype(np.float64))
    x = rng.standard_normal(P.field_shape)
    assert np.allclose(oracle_mod.apply(Pf, x), oracle_mod.apply(P, x), rtol=0, atol=1e-13)
    A, _ = oracle_mod.effective(P, tol=1e-13)
    Af, _ = oracle_mod.effective(Pf, tol=1e-13)
    assert np.allclose(Af, A, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("physics", [0, 1])
def test_uniform_fraction_gives_the_averaged_uniform_medium(oracle_mod, physics):
    """The same fraction f in every voxel is a uniform medium whose local operator
    is f M1 + (1 - f) M0, so A* = A0 + (f M1 + (1 - f) M0)^{-1} exactly (Gamma^h_0 = 0
    annihilates the constant polarisation)."""
    f = 0.3
    if physics == 1:
        mods = np.array([k_mu(1.0, 0.3), k_mu(10.0, 0.2)])
        ref = np.array(k_mu(0.4, 0.3))
        A0 = iso_mandel(*ref)
        A1, A2 = iso_mandel(*mods[0]), iso_mandel(*mods[1])
        shape = (6, 6, 6)
    else:
        mods = np.array([np.diag([1.0, 2.0]), np.diag([7.0, 5.0])])
        ref = 0.5 * np.eye(2)
        A0, A1, A2 = ref, mods[0], mods[1]
        shape = (8, 10)
    M = (1 - f) * np.linalg.inv(A1 - A0) + f * np.linalg.inv(A2 - A0)
    expected = A0 + np.linalg.inv(M)
    ph = np.zeros(shape, np.uint8)
    P = oracle_mod.Problem(ph, mods, physics=physics, green=oracle_mod.FILTERED, ref=ref,
                           frac=np.full(shape, f))
    A, _ = oracle_mod.effective(P, tol=1e-14)
    assert np.allclose(A, expected, rtol=1e-12, atol=1e-12)


def _golden_rows(name):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    rows = {}
    for line in open(path):
        line = line.split("#")[0].split()
        if line:
            rows[line[0]] = [float(v) for v in line[1:]]
    return rows


def test_default_reference_reproduces_the_papers_reference_medium(oracle_mod):
    """Sec. 5's table of mechanical parameters (tests/golden/sec5_mechanical_parameters.txt):
    from the matrix and inclusion entries, the default reference rule gives the table's
    reference medium (mu0 = mu_m / 2, nu0 = 0.3)."""
    rows = _golden_rows("sec5_mechanical_parameters.txt")

    def k_of(mu, nu):  # bulk modulus of an isotropic medium
        return 2.0 * mu * (1.0 + nu) / (3.0 * (1.0 - 2.0 * nu))

    moduli = np.array([[k_of(*rows["matrix"]), rows["matrix"][0]],
                       [k_of(*rows["inclusions"]), rows["inclusions"][0]]])
    K0, mu0 = oracle_mod.default_reference(3, oracle_mod.ELASTIC, moduli)
    mu_ref, nu_ref = rows["reference"]
    assert abs(mu0 - mu_ref) < 1e-14
    assert abs(K0 - k_of(mu_ref, nu_ref)) < 1e-13


# --------------------------------------------------------------------------- consistent operator (Eq. (11))
def _brute_consistent(k, N, a1, a2):
    """Eq. (11) summed literally over |n_i| <= L for L = 300, 600, 1200, then
    extrapolated (the truncated sums carry errors of order 1/L and 1/L^2)."""
    x = np.array(k, dtype=float) / N

    def trunc(L):
        n = np.arange(-L, L + 1)
        u, y = x[0] + n[:, None], x[1] + n[None, :]
        with np.errstate(divide="ignore", invalid="ignore"):
            w1 = np.where(u == 0, 1.0, np.sin(np.pi * x[0]) ** 2 / (np.pi * u) ** 2)
            w2 = np.where(y == 0, 1.0, np.sin(np.pi * x[1]) ** 2 / (np.pi * y) ** 2)
            q = a1 * u * u + a2 * y * y
            w = np.where(q == 0, 0.0, w1 * w2 / q)
        return np.array([[(w * u * u).sum(), (w * u * y).sum()], [(w * u * y).sum(), (w * y * y).sum()]])

    b1, b2, b4 = trunc(300), trunc(600), trunc(1200)
    r1, r2 = 2 * b2 - b1, 2 * b4 - b2
    return (4 * r2 - r1) / 3


def _consistent_problem(oracle_mod, N, A0, mods=None):
    ph = np.zeros((N, N), np.uint8)
    ph[N // 4:N // 2, N // 8:(5 * N) // 8] = 1
    mods = np.array([np.eye(2), 4.0 * np.eye(2)]) if mods is None else mods
    return oracle_mod.Problem(ph, mods, green=oracle_mod.CONSISTENT, ref=A0)


@pytest.mark.parametrize("A0", [np.diag([0.5, 0.5]), np.diag([0.5, 1.7])])
def test_consistent_operator_matches_the_lattice_sum(oracle_mod, A0):
    """The accelerated evaluation (closed-form inner lattice sums, Hurwitz tails) equals
    the series of Eq. (11) summed term by term."""
    N = 12
    P = _consistent_problem(oracle_mod, N, A0)
    for k in [(1, 1), (3, 5), (6, 6), (11, 2), (0, 4), (5, 0), (7, 9)]:
        G = np.real(oracle_mod.gamma_hat(P, k)).reshape(2, 2)
        assert np.abs(G - _brute_consistent(k, N, A0[0, 0], A0[1, 1])).max() < 1e-8, k


def test_consistent_operator_properties(oracle_mod):
    """Even and real in k; tr(A0 G_k) = 1 at every k != 0 (the weights F^2 sum to one
    and tr(A0 Gamma0) = 1); at low frequencies G_k -> Gamma0(k) as N grows, the gap
    shrinking like (k/N)^2; axis frequencies give Gamma0 exactly."""
    A0 = np.diag([0.5, 1.7])
    N = 16
    P = _consistent_problem(oracle_mod, N, A0)
    for k in [(1, 2), (3, 7), (5, 11), (8, 3)]:
        G = oracle_mod.gamma_hat(P, k)
        Gm = oracle_mod.gamma_hat(P, ((N - k[0]) % N, (N - k[1]) % N))
        assert np.abs(np.imag(G)).max() == 0.0
        assert np.allclose(G, Gm, atol=1e-13)
        Gr = np.real(G).reshape(2, 2)
        assert abs(np.trace(A0 @ Gr) - 1.0) < 1e-12
        assert np.allclose(Gr, Gr.T, atol=1e-15)
    g0 = lambda k: np.outer(k, k) / (np.asarray(k) @ A0 @ np.asarray(k))
    gaps = []
    for N in (16, 32, 64):
        P = _consistent_problem(oracle_mod, N, A0)
        gaps.append(np.abs(np.real(oracle_mod.gamma_hat(P, (1, 2))).reshape(2, 2) - g0([1, 2])).max())
    assert gaps[0] > gaps[1] > gaps[2] and 3.0 < gaps[0] / gaps[1] < 5.0 and 3.0 < gaps[1] / gaps[2] < 5.0
    Gx = np.real(oracle_mod.gamma_hat(P, (5, 0))).reshape(2, 2)
    assert np.allclose(Gx, g0([1, 0]), atol=1e-15)


def test_consistent_operator_galerkin_monotone_under_refinement(oracle_mod):
    """With the consistent operator, Eq. (13) is the exact Galerkin projection of the
    LS variational problem on piecewise-constant fields.  For A0 below both phases the
    form is coercive and A*_h p.p = A0 p.p + max over the subspace of a concave
    functional, so on nested grids (a grid-aligned square inclusion at N = 4, 8, 16) it
    increases with N and stays below the Voigt bound; CG equals the dense solve of
    Eq. (12) (N = 4); the filtered and truncated operators approach the same values as N
    grows."""
    mods = np.array([np.eye(2), 10.0 * np.eye(2)])
    A0 = 0.5 * np.eye(2)
    e1 = np.array([1.0, 0.0])
    vals = {}
    for N in (4, 8, 16):
        ph = ms.square_inclusion(N)
        for green in (oracle_mod.CONSISTENT, oracle_mod.FILTERED, oracle_mod.TRUNCATED):
            P = oracle_mod.Problem(ph, mods, green=green, ref=A0)
            tau, _, _ = oracle_mod.solve(P, e1, tol=1e-14, solver=1)
            vals[(green, N)] = A0[0, 0] + tau[0].mean()  # e1 . A*_h e1, Eq. (tau_Astar)
            if N == 4 and green == oracle_mod.CONSISTENT:
                assert np.allclose(tau, oracle_mod.dense_solve(P, e1), atol=1e-11)
                assert abs(tau[1].mean()) < 1e-13  # A*_12 = 0 by the square's symmetry
    c = oracle_mod.CONSISTENT
    assert vals[(c, 4)] < vals[(c, 8)] < vals[(c, 16)] < 0.75 * 1.0 + 0.25 * 10.0
    for green in (oracle_mod.FILTERED, oracle_mod.TRUNCATED):
        assert abs(vals[(green, 16)] - vals[(c, 16)]) < abs(vals[(green, 4)] - vals[(c, 4)])


def test_consistent_operator_refuses_what_it_does_not_cover(oracle_mod):
    """Elastic problems, 3D and non-diagonal references are outside its scope."""
    ph = np.zeros((6, 6), np.uint8)
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.effective(oracle_mod.Problem(ph, np.array([2.0 * np.eye(2)]), green=oracle_mod.CONSISTENT,
                                                ref=np.array([[1.0, 0.2], [0.2, 1.0]])), tol=1e-10)
    ph3 = np.zeros((4, 4, 4), np.uint8)
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.effective(oracle_mod.Problem(ph3, np.array([2.0 * np.eye(3)]), green=oracle_mod.CONSISTENT,
                                                ref=np.eye(3)), tol=1e-10)
