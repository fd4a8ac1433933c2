"""Pins of the oracle's time reversal Theta = exp(-i pi S^y) K (Sec. II.B: the
time-reversal symmetry behind the pairs of mutually time-reversed random
vectors, tau = 1 in Sec. III) against its definition and its algebra."""
import numpy as np
import pytest
from conftest import oracle_system, random_system

import oracle
from oracle import dense


@pytest.mark.parametrize("two_s", [[1, 1, 1], [2, 1, 3], [5, 4], [1, 2, 4, 1]])
def test_matches_exponential_of_sy(two_s, rng):
    """Theta x = (x)_i expm(-i pi s^y_i) conj(x), the definition, built with
    scipy's matrix exponential."""
    w = random_system(rng, two_s)
    s = oracle_system(w)
    x = rng.normal(size=(s.dim, 3)) + 1j * rng.normal(size=(s.dim, 3))
    U = dense.time_reversal_unitary(two_s)
    assert np.allclose(oracle.time_reverse(s, x), U @ x.conj(), atol=1e-12)


@pytest.mark.parametrize("two_s", [[1, 1, 1], [1, 1], [2, 1, 3], [2, 2], [5, 4, 1]])
def test_kramers(two_s, rng):
    """Theta^2 = (-1)^(2 S_max): -1 for half-integer total spin, +1 otherwise."""
    w = random_system(rng, two_s)
    s = oracle_system(w)
    x = rng.normal(size=s.dim) + 1j * rng.normal(size=s.dim)
    sign = -1.0 if sum(two_s) % 2 else 1.0
    assert np.allclose(oracle.time_reverse(s, oracle.time_reverse(s, x)), sign * x, atol=1e-13)


def test_antiunitary(rng):
    """<Theta a|Theta b> = conj <a|b>."""
    w = random_system(rng, [2, 3, 1])
    s = oracle_system(w)
    a = rng.normal(size=s.dim) + 1j * rng.normal(size=s.dim)
    b = rng.normal(size=s.dim) + 1j * rng.normal(size=s.dim)
    ta, tb = oracle.time_reverse(s, a), oracle.time_reverse(s, b)
    assert np.isclose(np.vdot(ta, tb), np.conj(np.vdot(a, b)), atol=1e-12)


def test_reverses_the_field(rng):
    """Theta H(B) Theta^-1 = H(-B): Eq. 3's exchange, single-ion and dipolar
    terms are even in the spins, the Zeeman term odd.  So Lanczos from Theta r
    with field B gives the alpha, beta of Lanczos from r with field -B, and
    <Theta r|H(B)|Theta r> = <r|H(-B)|r>."""
    w = random_system(rng, [1, 2, 3, 1])
    s = oracle_system(w)
    wm = dict(w, B=-np.asarray(w["B"]))
    sm = oracle_system(wm)
    r = rng.normal(size=s.dim) + 1j * rng.normal(size=s.dim)
    r /= np.linalg.norm(r)
    tr = oracle.time_reverse(s, r)
    assert np.isclose(np.vdot(tr, oracle.apply_h(s, tr)), np.vdot(r, oracle.apply_h(sm, r)), atol=1e-11)
    a1, b1, _, m1 = oracle.lanczos(s, tr, 12)
    a2, b2, _, m2 = oracle.lanczos(sm, r, 12)
    assert m1 == m2
    assert np.allclose(a1[:m1], a2[:m2], atol=1e-10) and np.allclose(b1[:m1 - 1], b2[:m2 - 1], atol=1e-10)


def test_zero_field_commutes(rng):
    """B = 0: Theta commutes with H (Kramers pairs of the spectrum for
    half-integer total spin)."""
    w = dict(random_system(rng, [1, 1, 3]), B=np.zeros(3))
    s = oracle_system(w)
    x = rng.normal(size=s.dim) + 1j * rng.normal(size=s.dim)
    assert np.allclose(oracle.apply_h(s, oracle.time_reverse(s, x)), oracle.time_reverse(s, oracle.apply_h(s, x)),
                       atol=1e-11)
    ev = np.linalg.eigvalsh(dense.hamiltonian(s))
    assert np.allclose(ev[0::2], ev[1::2], atol=1e-9)  # every level twice


def test_pairs_start_block(rng):
    """The pairs block: even global vectors are the plain random vectors
    v // 2, odd ones their time reverses; a pair is orthogonal in the
    Hermitian product's real part, and both are unit vectors."""
    w = random_system(rng, [2, 1, 2])
    s = oracle_system(w)
    P = oracle.start_pairs(s, 6, seed=9, vec_offset=4)
    base = oracle.start_vectors(s.dim, 3, seed=9, vec_offset=2)
    assert np.allclose(P[:, 0::2], base, atol=1e-15)
    assert np.allclose(P[:, 1::2], oracle.time_reverse(s, base), atol=1e-15)
    assert np.allclose(np.linalg.norm(P, axis=0), 1.0)


def test_ftlm_pairs_runs_reverse_field(rng):
    """In a pairs run the odd vectors' tridiagonal data equal those of the
    even vectors with the field reversed (alpha, beta; p changes sign with
    the observable u.S, which is odd under Theta)."""
    w = random_system(rng, [1, 2, 1, 1])
    s = oracle_system(w)
    wm = dict(w, B=-np.asarray(w["B"]))
    sm = oracle_system(wm)
    u = np.asarray(w["B"]) / np.linalg.norm(w["B"])
    T = oracle.default_temperatures()
    g = oracle.ftlm(s, R=4, M=10, T=T, seed=3, start="pairs", direction=u)
    h = oracle.ftlm(sm, R=2, M=10, T=T, seed=3, start="random", direction=u)
    assert np.allclose(g["alpha"][1::2], h["alpha"], atol=1e-10)
    assert np.allclose(g["beta"][1::2, :9], h["beta"][:, :9], atol=1e-10)
    assert np.allclose(g["p"][1::2], -np.conj(h["p"]), atol=1e-10)
