"""Test-side helpers: material constants and closed forms written from textbook
mechanics, independent of both the oracle and the CUDA path."""
import numpy as np

SQ2 = np.sqrt(2.0)
MANDEL = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def k_mu(E, nu):
    """(bulk, shear) from Young's modulus and Poisson's ratio."""
    return E / (3.0 * (1.0 - 2.0 * nu)), E / (2.0 * (1.0 + nu))


def iso_stiffness_tensor(K, mu):
    lam = K - 2.0 * mu / 3.0
    d = np.eye(3)
    return (lam * np.einsum("ij,kl->ijkl", d, d)
            + mu * (np.einsum("ik,jl->ijkl", d, d) + np.einsum("il,jk->ijkl", d, d)))


def tensor4_to_mandel(C):
    M = np.zeros((6, 6))
    for I, (i, j) in enumerate(MANDEL):
        for J, (k, l) in enumerate(MANDEL):
            M[I, J] = (1 if I < 3 else SQ2) * (1 if J < 3 else SQ2) * C[i, j, k, l]
    return M


def mandel_to_tensor2(v):
    T = np.zeros((3, 3))
    for I, (i, j) in enumerate(MANDEL):
        val = v[I] if I < 3 else v[I] / SQ2
        T[i, j] = T[j, i] = val
    return T


def tensor2_to_mandel(T):
    return np.array([T[i, j] if I < 3 else SQ2 * T[i, j] for I, (i, j) in enumerate(MANDEL)])


def iso_mandel(K, mu):
    return tensor4_to_mandel(iso_stiffness_tensor(K, mu))


def laminate_elastic(Cs, fracs, axis):
    """Effective stiffness (Mandel) of a laminate with layer normal e_axis.

    Continuity of the in-plane strain components and of the traction sigma.n
    across layers: split Mandel components into those that involve the
    normal index (N) and the others (T).  With uniform eps_T and sigma_N:
      eps_N = C_NN^{-1} (sigma_N - C_NT eps_T) per layer,
      sigma_N = <C_NN^{-1}>^{-1} (E_N + <C_NN^{-1} C_NT> E_T),
      <sigma_T> = <C_TN eps_N> + <C_TT> E_T.
    """
    Nset = [I for I, (i, j) in enumerate(MANDEL) if axis in (i, j)]
    Tset = [I for I in range(6) if I not in Nset]
    inv_nn = sum(f * np.linalg.inv(C[np.ix_(Nset, Nset)]) for C, f in zip(Cs, fracs))
    inv_nn_nt = sum(f * np.linalg.inv(C[np.ix_(Nset, Nset)]) @ C[np.ix_(Nset, Tset)] for C, f in zip(Cs, fracs))
    A = np.linalg.inv(inv_nn)  # sigma_N = A E_N + A inv_nn_nt E_T
    Ceff = np.zeros((6, 6))
    # columns for unit macroscopic strains
    for J in range(6):
        E = np.zeros(6)
        E[J] = 1.0
        EN, ET = E[Nset], E[Tset]
        SN = A @ (EN + inv_nn_nt @ ET)
        sT = np.zeros(len(Tset))
        for C, f in zip(Cs, fracs):
            eN = np.linalg.solve(C[np.ix_(Nset, Nset)], SN - C[np.ix_(Nset, Tset)] @ ET)
            sT += f * (C[np.ix_(Tset, Nset)] @ eN + C[np.ix_(Tset, Tset)] @ ET)
        Ceff[Nset, J] = SN
        Ceff[Tset, J] = sT
    return Ceff


def hs_bounds_2d(k1, k2, f2):
    """Hashin-Shtrikman bounds for an isotropic 2D two-phase conductor, k1 < k2."""
    f1 = 1.0 - f2
    lo = k1 + f2 / (1.0 / (k2 - k1) + f1 / (2.0 * k1))
    hi = k2 + f1 / (1.0 / (k1 - k2) + f2 / (2.0 * k2))
    return lo, hi


def hs_bounds_elastic(K1, mu1, K2, mu2, f2):
    """Hashin-Shtrikman bounds on (K*, mu*) for an isotropic 3D two-phase
    composite with phase 1 the softer one (K1 <= K2, mu1 <= mu2)."""
    f1 = 1.0 - f2
    Klo = K1 + f2 / (1.0 / (K2 - K1) + 3.0 * f1 / (3.0 * K1 + 4.0 * mu1))
    Khi = K2 + f1 / (1.0 / (K1 - K2) + 3.0 * f2 / (3.0 * K2 + 4.0 * mu2))
    mulo = mu1 + f2 / (1.0 / (mu2 - mu1) + 6.0 * f1 * (K1 + 2 * mu1) / (5.0 * mu1 * (3 * K1 + 4 * mu1)))
    muhi = mu2 + f1 / (1.0 / (mu1 - mu2) + 6.0 * f2 * (K2 + 2 * mu2) / (5.0 * mu2 * (3 * K2 + 4 * mu2)))
    return (Klo, Khi), (mulo, muhi)


def iso_projection(C):
    """(K, mu) of the isotropic part of a Mandel stiffness."""
    J = np.zeros((6, 6))
    J[:3, :3] = 1.0 / 3.0
    Kdev = np.eye(6) - J
    K = np.trace(J @ C) / 3.0
    mu = np.trace(Kdev @ C) / 10.0
    return K, mu
