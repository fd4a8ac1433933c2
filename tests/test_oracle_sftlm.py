"""Pins of the oracle's symmetric FTLM (Eqs. E-2-G, E-2-H) for O = u.S:
against the definition-level traces, the single-vector expectation value
evaluated with dense matrix functions, the commuting case and the FTLM
projections."""
import numpy as np
import pytest
from conftest import oracle_system, random_system

import oracle
from oracle import dense

T = np.array([0.1, 0.3, 1.0, 3.0, 10.0, 30.0])


def test_all_basis_vectors_full_krylov_is_exact(rng):
    """R = d basis vectors, M = d with full re-orthogonalisation: the sums of
    Eq. (E-2-G) become Tr(e^{-bH/2} O e^{-bH/2}) / Tr(e^{-bH}) = <O>, the
    exact thermal average (from the ED of the Kronecker-product H)."""
    w = random_system(rng, [2, 1, 3])  # d = 24
    s = oracle_system(w)
    u = np.array([0.3, -0.2, 0.9]) / np.linalg.norm([0.3, -0.2, 0.9])
    o = oracle.sftlm(s, R=s.dim, M=s.dim, T=T, start="basis", reorth=True, direction=u)
    ex = dense.thermo_exact(s, T, direction=u)
    assert np.max(np.abs(o["M_B_sym"] - ex["M_B"])) < 1e-10 * max(1.0, np.abs(ex["M_B"]).max())
    assert np.max(np.abs(o["M_B_sym_imag"])) < 1e-10


def test_single_vector_matches_matrix_functions(rng):
    """One random vector, full Krylov space: (E-2-H) equals
    <r|e^{-bH/2} O e^{-bH/2}|r> / <r|e^{-bH}|r> from the dense eigendecomposition."""
    w = random_system(rng, [1, 2, 1, 1])  # d = 24
    s = oracle_system(w)
    u = np.asarray(w["B"]) / np.linalg.norm(w["B"])
    o = oracle.sftlm(s, R=1, M=s.dim, T=T, seed=4, reorth=True, direction=u)
    assert o["M_eff"][0] == s.dim
    r = oracle.start_vectors(s.dim, 1, seed=4)[:, 0]
    H = dense.hamiltonian(s)
    Ou = dense.total_spin_along(s, u)
    ev, V = np.linalg.eigh(H)
    c = V.conj().T @ r
    for k, t in enumerate(T):
        half = V @ (np.exp(-(ev - ev[0]) / (2 * t)) * c)   # e^{-bH/2}|r> up to e^{b E0/2}
        num = np.vdot(half, Ou @ half)
        den = np.vdot(half, half).real
        assert abs(o["M_B_sym"][k] - (-w["g"] * num.real / den)) < 1e-9 * max(1.0, abs(num.real / den))


def test_commuting_observable_equals_ftlm(rng):
    """[H, u.S] = 0 (isotropic exchange, Zeeman along u, no anisotropy or
    dipolar term): the symmetric and asymmetric forms of Eq. (E-2-F) agree.
    Each run goes to the end of its Krylov space (re-orthogonalised, until
    breakdown), where both Krylov sums are the exact expectation values."""
    n = 4
    J = np.zeros((n, n))
    for i in range(n - 1):
        J[i, i + 1] = rng.uniform(0.5, 1.5)
    w = {"two_s": np.array([1, 2, 1, 3]), "J": J, "d_ion": None, "e_axes": None, "g": 2.0,
         "B": np.array([0.0, 0.0, 0.7]), "pos": None}
    s = oracle_system(w)
    o = oracle.sftlm(s, R=3, M=s.dim, T=T, seed=1, reorth=True, tol=1e-10)
    assert np.allclose(o["M_B_sym"], o["M_B"], rtol=1e-9, atol=1e-11)
    # and an anisotropic system does not (the point of Eq. E-2-G)
    w2 = random_system(rng, [1, 2, 1, 3])
    s2 = oracle_system(w2)
    o2 = oracle.sftlm(s2, R=3, M=8, T=T, seed=1)
    assert np.max(np.abs(o2["M_B_sym"] - o2["M_B"])) > 1e-4


def test_projection_matrix(rng):
    """O_ij = <v_i|O|v_j> is Hermitian and its first column is the FTLM
    projection p_j = <v_j|O|v_0>."""
    w = random_system(rng, [2, 2, 1])
    s = oracle_system(w)
    o = oracle.sftlm(s, R=2, M=10, T=T, seed=2)
    f = oracle.ftlm(s, R=2, M=10, T=T, seed=2)
    for r in range(2):
        m = o["M_eff"][r]
        O = o["O"][r, :m, :m]
        assert np.allclose(O, O.conj().T, atol=1e-12)
        assert np.allclose(O[:, 0], f["p"][r, :m], atol=1e-12)
    for k in ("lnZ", "E", "C", "M_B"):
        assert np.allclose(o[k], f[k], rtol=1e-12)


def test_sums_reproduce_driver(rng):
    w = random_system(rng, [1, 1, 2, 1])
    s = oracle_system(w)
    o = oracle.sftlm(s, R=3, M=12, T=T, seed=6, start="pairs")
    mb, mbi = oracle.sftlm_sums(o["alpha"], o["beta"], o["O"], o["M_eff"], w["g"], T)
    assert np.allclose(mb, o["M_B_sym"], rtol=1e-13) and np.allclose(mbi, o["M_B_sym_imag"], atol=1e-13)
