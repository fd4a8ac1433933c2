"""Pins for the Hamiltonian of Eq. (3): the definition-level builder
(``oracle.dense``) against closed forms, and the oracle's ladder-form column
scatter against the definition-level builder."""
import numpy as np
import pytest
from conftest import oracle_system, random_system

import ftlm_workloads as W
import oracle
from oracle import dense

MU_B, C_DIP = oracle.MU_B_DEFAULT, oracle.C_DIP_DEFAULT


@pytest.mark.parametrize("two_s", [1, 2, 3, 4, 5])
def test_spin_algebra(two_s):
    sx, sy, sz = dense.spin_matrices(two_s)
    s = two_s / 2
    assert np.allclose(sx @ sy - sy @ sx, 1j * sz)
    assert np.allclose(sy @ sz - sz @ sy, 1j * sx)
    assert np.allclose(sx @ sx + sy @ sy + sz @ sz, s * (s + 1) * np.eye(two_s + 1))


def _single(two_s, **kw):
    w = {"two_s": [two_s], "J": np.zeros((1, 1)), "g": 2.0, "B": np.zeros(3)}
    w.update(kw)
    return oracle.System(**w)


@pytest.mark.parametrize("two_s", [1, 2, 5])
def test_zeeman_spectrum(two_s, rng):
    B = rng.normal(size=3)
    s = _single(two_s, B=B)
    ev = np.linalg.eigvalsh(dense.hamiltonian(s))
    m = np.arange(two_s + 1) - two_s / 2
    assert np.allclose(ev, np.sort(MU_B * 2.0 * np.linalg.norm(B) * m))


@pytest.mark.parametrize("two_s", [1, 2, 5])
def test_single_ion_spectrum(two_s, rng):
    e = rng.normal(size=3)
    s = _single(two_s, d_ion=[-3.0], e_axes=[e])
    ev = np.linalg.eigvalsh(dense.hamiltonian(s))
    m = np.arange(two_s + 1) - two_s / 2
    assert np.allclose(ev, np.sort(-3.0 * m ** 2))


def test_dipolar_dimer_closed_form(rng):
    """Two s=1/2 at distance r, any orientation: H_dip = C g^2/r^3 (s1.s2 - 3(s1.e)(e.s2))
    has eigenvalues C g^2/r^3 * {-1/2, -1/2, 0, 1}."""
    rv = rng.normal(size=3)
    r = np.linalg.norm(rv)
    s = oracle.System(two_s=[1, 1], J=np.zeros((2, 2)), g=2.0, B=np.zeros(3), pos=np.stack([np.zeros(3), rv]))
    ev = np.linalg.eigvalsh(dense.hamiltonian(s))
    assert np.allclose(ev, np.sort(C_DIP * 4.0 / r ** 3 * np.array([-0.5, -0.5, 0.0, 1.0])))


@pytest.mark.parametrize("two_s", [1, 2, 3])
def test_heisenberg_dimer_levels(two_s):
    """2 J s1.s2 = J [S(S+1) - 2 s(s+1)], S = 0..2s with 2S+1 states each, plus
    a field along z shifting by g mu_B B M_S."""
    J, B = 0.7, 0.3
    s = oracle.System(two_s=[two_s, two_s], J=np.array([[0, J], [0, 0]]), g=2.0, B=[0, 0, B])
    ev = np.linalg.eigvalsh(dense.hamiltonian(s))
    sv = two_s / 2
    ref = [J * (S * (S + 1) - 2 * sv * (sv + 1)) + 2.0 * MU_B * B * M
           for S in range(two_s + 1) for M in np.arange(-S, S + 1)]
    assert np.allclose(ev, np.sort(ref))


def test_trace_identities(rng):
    two_s = [1, 2, 3]
    S = dense.site_operators(two_s)
    d = 2 * 3 * 4
    for i in range(3):
        for j in range(3):
            t = sum((S[i][a] @ S[j][a]).diagonal().sum() for a in range(3))
            if i != j:
                assert abs(t) < 1e-12
        e = rng.normal(size=3)
        e /= np.linalg.norm(e)
        se = sum(e[a] * S[i][a] for a in range(3))
        s = two_s[i] / 2
        assert np.isclose((se @ se).diagonal().sum().real, d * s * (s + 1) / 3)
    # hence tr H = d sum_i d_i s_i (s_i + 1) / 3 (exchange, dipolar, Zeeman are traceless)
    w = random_system(rng, two_s)
    sysm = oracle_system(w)
    H = dense.hamiltonian(sysm)
    ss = np.array(two_s) / 2
    assert np.isclose(np.trace(H).real, d * np.sum(w["d_ion"] * ss * (ss + 1) / 3))


def test_spin_half_single_ion_is_constant(rng):
    n = 3
    d_ion = rng.normal(size=n)
    s = oracle.System(two_s=[1] * n, J=np.zeros((n, n)), B=np.zeros(3), d_ion=d_ion, e_axes=rng.normal(size=(n, 3)))
    H = dense.hamiltonian(s)
    assert np.allclose(H, d_ion.sum() / 4 * np.eye(8))


def _rotation(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return q * np.sign(np.linalg.det(q))


def test_global_rotation_and_time_reversal_keep_spectrum(rng):
    w = random_system(rng, [1, 2, 1, 3])
    s0 = oracle_system(w)
    ev0 = np.linalg.eigvalsh(dense.hamiltonian(s0))
    Rm = _rotation(rng)
    w2 = dict(w, pos=w["pos"] @ Rm.T, e_axes=w["e_axes"] @ Rm.T, B=Rm @ w["B"])
    assert np.allclose(np.linalg.eigvalsh(dense.hamiltonian(oracle_system(w2))), ev0)
    w3 = dict(w, B=-w["B"])
    assert np.allclose(np.linalg.eigvalsh(dense.hamiltonian(oracle_system(w3))), ev0)


# --- the oracle's ladder-form matvec against the definition -------------------

CASES = {
    "mixed": lambda rng: random_system(rng, [1, 2, 3, 5]),
    "spin1_ring6": lambda rng: W.ring6_s1(),
    "half_4x3": lambda rng: W.square_lattice(4, 3, seed=1),
    "half_12_random": lambda rng: random_system(rng, [1] * 12),
    "spin32_6": lambda rng: random_system(rng, [3] * 6, scale=5.0),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_oracle_matvec_matches_definition(case, rng):
    s = oracle_system(CASES[case](rng))
    H = dense.hamiltonian_sparse(s)
    X = rng.normal(size=(s.dim, 3)) + 1j * rng.normal(size=(s.dim, 3))
    Y = oracle.apply_h(s, X)
    ref = H @ X
    assert np.linalg.norm(Y - ref) <= 1e-13 * np.linalg.norm(ref)
    assert abs(H - H.conj().T).max() < 1e-12


def test_oracle_columns_and_rows(rng):
    s = oracle_system(random_system(rng, [1, 2, 1, 3, 1]))
    H = dense.hamiltonian(s)
    for nu in rng.integers(0, s.dim, size=8):
        rows, vals = oracle.h_column(s, int(nu))
        col = np.zeros(s.dim, dtype=complex)
        col[rows] = vals
        assert np.allclose(col, H[:, nu], atol=1e-13)
    X = rng.normal(size=(s.dim, 2)) + 1j * rng.normal(size=(s.dim, 2))
    mus = rng.integers(0, s.dim, size=10)
    assert np.allclose(oracle.h_rows(s, mus, X), (H @ X)[mus], atol=1e-12)


def test_oracle_hermitian_large(rng):
    """<x|H y> = conj(<y|H x>) at d = 65,536 with all-pairs dipolar coupling."""
    s = oracle_system(W.lattice4x4())
    x = rng.normal(size=s.dim) + 1j * rng.normal(size=s.dim)
    y = rng.normal(size=s.dim) + 1j * rng.normal(size=s.dim)
    a = np.vdot(x, oracle.apply_h(s, y))
    b = np.vdot(y, oracle.apply_h(s, x))
    assert abs(a - np.conj(b)) <= 1e-12 * abs(a)


def test_oracle_total_spin(rng):
    s = oracle_system(random_system(rng, [1, 2, 3]))
    u = rng.normal(size=3)
    O = dense.total_spin_along(s, u)
    X = rng.normal(size=(s.dim, 2)) + 1j * rng.normal(size=(s.dim, 2))
    assert np.allclose(oracle.apply_sdir(s, u, X), O @ X, atol=1e-13)


def test_dodecahedron_directions():
    """The powder-average directions with their antipodes are the 20 vertices
    of a regular dodecahedron: unit vectors, and the shortest distance between
    two of them occurs exactly 30 times (the 30 edges)."""
    import ftlm_workloads as W
    u = W.dodecahedron_directions()
    v = np.concatenate([u, -u])
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0)
    dist = np.linalg.norm(v[:, None, :] - v[None, :, :], axis=2)
    iu = np.triu_indices(20, 1)
    dd = dist[iu]
    assert np.sum(np.isclose(dd, dd.min())) == 30 and dd.min() > 0.5
