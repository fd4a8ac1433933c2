"""Pins for the oracle's Lanczos recurrence, tridiagonal eigensolver and the
FTLM sums of Eqs. (4)-(5): library eigensolvers, moment identities, exact
diagonalisation when the Krylov space is complete, and closed forms."""
import numpy as np
import pytest
from conftest import oracle_system, random_system

import ftlm_workloads as W
import oracle
from oracle import dense

T = W.temperatures()
MU_B = oracle.MU_B_DEFAULT


def _rel(a, b, floor_frac=1e-3):
    """Relative error with a floor of floor_frac * max|b| (quantities that pass through 0)."""
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b) / np.maximum(np.abs(b), floor_frac * np.max(np.abs(b))))


def test_jacobi_matches_lapack(rng):
    for m in (1, 2, 7, 40):
        a = rng.normal(size=m)
        b = np.abs(rng.normal(size=m))
        ev, U = oracle.tridiag_eig(a, b)
        Tm = np.diag(a) + np.diag(b[: m - 1], 1) + np.diag(b[: m - 1], -1)
        w, V = np.linalg.eigh(Tm)
        order = np.argsort(ev)
        assert np.allclose(ev[order], w, atol=1e-13)
        assert np.allclose(np.abs(U[0, order]), np.abs(V[0]), atol=1e-10)
        assert np.allclose(U.T @ U, np.eye(m), atol=1e-13)
        assert np.allclose(Tm @ U, U * ev, atol=1e-12)


def test_lanczos_moments(rng):
    """sum_n |U_0n|^2 eps_n^k = <v0|H^k|v0> for k <= 2M-1 (Gauss quadrature)."""
    s = oracle_system(random_system(rng, [1, 2, 1, 2, 1]))
    H = dense.hamiltonian(s)
    v0 = rng.normal(size=s.dim) + 1j * rng.normal(size=s.dim)
    v0 /= np.linalg.norm(v0)
    M = 6
    a, b, p, m = oracle.lanczos(s, v0, M)
    assert m == M
    ev, U = oracle.tridiag_eig(a, b)
    w = U[0] ** 2
    assert np.isclose(w.sum(), 1.0, atol=1e-14)
    x = v0.copy()
    scale = np.abs(ev).max()
    for k in range(2 * M):
        mom = np.vdot(v0, x).real
        assert np.isclose((w * ev ** k).sum() / scale ** k, mom / scale ** k, atol=1e-11), k
        x = H @ x


def test_lanczos_projection(rng):
    """p_j = <v_j | (u.S) v0>; with one step p_0 = <v0|u.S|v0>, and
    sum_j U_jn conj(p_j) = <v0|u.S|n> for the Ritz vectors n."""
    s = oracle_system(random_system(rng, [2, 1, 2]))
    u = dense.field_direction(s)
    O = dense.total_spin_along(s, u)
    H = dense.hamiltonian(s)
    v0 = rng.normal(size=s.dim) + 1j * rng.normal(size=s.dim)
    v0 /= np.linalg.norm(v0)
    a, b, p, m = oracle.lanczos(s, v0, 1)
    assert np.isclose(p[0], np.vdot(v0, O @ v0))
    a, b, p, m = oracle.lanczos(s, v0, 5, reorth=True)
    # rebuild the Lanczos vectors from the recurrence with the dense H
    V = [v0]
    w = H @ v0 - a[0] * v0
    for j in range(1, 5):
        V.append(w / b[j - 1])
        w = H @ V[j] - a[j] * V[j] - b[j - 1] * V[j - 1]
    V = np.array(V).T
    for j in range(5):
        assert np.isclose(p[j], np.vdot(V[:, j], O @ v0), atol=1e-12)


@pytest.mark.parametrize("two_s", [[1] * 6, [2, 2, 2, 2], [1, 3, 2]])
def test_exact_mode_all_basis_vectors_equals_ed(two_s, rng):
    """FTLM on all d basis vectors with full Krylov depth (and full
    re-orthogonalisation) reproduces exact diagonalisation."""
    s = oracle_system(random_system(rng, two_s))
    d = s.dim
    r = oracle.ftlm(s, R=d, M=d, T=T, start="basis", reorth=True)
    ex = dense.thermo_exact(s, T)
    for k in ("lnZ", "E", "C", "M_B"):
        assert _rel(r[k], ex[k], 1e-6) < 1e-10, k
    assert np.abs(r["M_B_imag"]).max() < 1e-10 * np.abs(ex["M_B"]).max()


@pytest.mark.slow
def test_exact_mode_on_the_s1_ring_equals_ed():
    """The same at d = 243: a ring of five s = 1 sites with every term of
    Eq. (3) (the model of the N = 6 ring, one site fewer).  243 start vectors
    x 243 steps with full re-orthogonalisation and 243 Jacobi eigensolves of
    order 243 (about 20 s on eight host threads).  The N = 6 ring itself
    (d = 729) costs about 40 s per Jacobi eigensolve, i.e. hours for the 729
    start vectors; it is checked by the next test."""
    s = oracle_system(W.ring(N=5, two_s=2))
    d = s.dim
    r = oracle.ftlm(s, R=d, M=d, T=T, start="basis", reorth=True)
    ex = dense.thermo_exact(s, T)
    for k in ("lnZ", "E", "C", "M_B"):
        assert _rel(r[k], ex[k], 1e-6) < 1e-10, k


@pytest.mark.slow
def test_ring6_all_basis_vectors_full_depth_equals_ed():
    """The N = 6, s = 1 ring (d = 729, tilted axes, oblique field, dipolar
    coupling): the oracle's three-term recurrence (no re-orthogonalisation,
    as on the hot path) from each of the 729 basis vectors, 729 steps deep.
    With the Krylov space complete, Eqs. (4)-(5) over all basis vectors are
    the exact traces Tr(e^{-H/T}), Tr(H e^{-H/T}), Tr(u.S e^{-H/T}); the
    eigenpairs of each tridiagonal matrix come from LAPACK's tridiagonal
    solver here, since the oracle's Jacobi takes about 40 s at order 729.
    Against exact diagonalisation of the dense Hamiltonian, within 1e-10
    (about 90 s on eight host threads).  d = 4096 would cost
    (4096/729)^3 = 177 times the recurrence work: out of reach on the CPU."""
    from scipy.linalg import eigh_tridiagonal
    w = W.ring6_s1()
    s = oracle_system(w)
    d = s.dim
    r = oracle.ftlm_tridiag(s, R=d, M=d, start="basis")
    assert np.all(r["M_eff"] == d)                      # every Krylov space is the whole space
    ev_all, u0_all, q_all = [], [], []
    for k in range(d):
        ev, U = eigh_tridiagonal(r["alpha"][k], r["beta"][k, : d - 1])
        ev_all.append(ev)
        u0_all.append(U[0])
        q_all.append(U.T @ np.conj(r["p"][k]))          # <r|u.S|n> = sum_j U_jn conj(p_j)
    ev, u0, q = np.array(ev_all), np.array(u0_all), np.array(q_all)
    E0 = ev.min()
    g = float(w["g"])
    res = {k: np.empty(len(T)) for k in ("lnZ", "E", "C", "M_B")}
    for t, Tk in enumerate(T):                           # Eqs. (4), (5) with R = d, prefactor d / R = 1
        bz = np.exp(-(ev - E0) / Tk)
        wgt = u0 ** 2 * bz
        z = wgt.sum()
        Em = (wgt * ev).sum() / z
        res["lnZ"][t] = np.log(z) - E0 / Tk
        res["E"][t] = Em
        res["C"][t] = (wgt * (ev - Em) ** 2).sum() / z / Tk ** 2
        res["M_B"][t] = -g * (bz * u0 * q).sum().real / z
    ex = dense.thermo_exact(s, T)
    for k in res:
        assert _rel(res[k], ex[k], 1e-6) < 1e-10, k


def test_exact_krylov_random_vectors_equals_trace_estimate(rng):
    """With the Krylov space complete, the FTLM estimate for fixed random
    vectors equals the exact stochastic trace sum_r <r|f(H)|r> (Eqs. 1, 4, 5)."""
    w = W.ring(N=5, two_s=2)       # d = 243, every term of Eq. (3)
    s = oracle_system(w)
    d, R = s.dim, 3
    r = oracle.ftlm(s, R=R, M=d, T=T, seed=11, reorth=True)
    vecs = oracle.start_vectors(d, R, seed=11)
    ex = dense.thermo_from_vectors(s, T, vecs)
    for k in ("lnZ", "E", "C", "M_B", "M_B_imag"):
        floor = 1e-6 if k != "M_B_imag" else 1.0
        assert _rel(r[k], ex[k], floor) < 1e-9, k


def test_zeeman_only_closed_form():
    """J = d = 0, no dipolar: Z = prod_i sinh((2s+1)x/2)/sinh(x/2), x = beta g mu_B |B|;
    M_B = g sum_i s B_s(s x) (Brillouin), E and C from d ln Z / d beta."""
    two_s = [1, 2, 3]
    B = np.array([0.3, -0.4, 1.2])
    g = 2.0
    s = oracle.System(two_s=two_s, J=np.zeros((3, 3)), g=g, B=B)
    h = g * MU_B * np.linalg.norm(B)
    lnZ = np.zeros(len(T)); E = np.zeros(len(T)); C = np.zeros(len(T)); M = np.zeros(len(T))
    for t2 in two_s:
        sv = t2 / 2
        x = h / T
        a = (2 * sv + 1) * x / 2
        lnZ += np.log(np.sinh(a) / np.sinh(x / 2))
        mean_m = -((2 * sv + 1) / 2 / np.tanh(a) - 0.5 / np.tanh(x / 2))
        var_m = -((2 * sv + 1) ** 2 / 4 / np.sinh(a) ** 2) + 0.25 / np.sinh(x / 2) ** 2
        E += h * mean_m
        C += x ** 2 * var_m
        M += -g * mean_m
    r = oracle.ftlm(s, R=s.dim, M=s.dim, T=T, start="basis", reorth=True)
    assert _rel(r["lnZ"], lnZ) < 1e-10
    assert _rel(r["E"], E) < 1e-10
    assert _rel(r["C"], C, 1e-6) < 1e-9
    assert _rel(r["M_B"], M) < 1e-10
    ex = dense.thermo_exact(s, T)
    assert _rel(ex["M_B"], M) < 1e-10 and _rel(ex["lnZ"], lnZ) < 1e-10


def test_decoupled_sites_factorise(rng):
    """J = 0, no dipolar, arbitrary d_i, e_i, B: Z = prod_i Z_i (single-site ED)."""
    w = random_system(rng, [2, 3, 1], dipolar=False)
    w["J"] = np.zeros((3, 3))
    s = oracle_system(w)
    r = oracle.ftlm(s, R=s.dim, M=s.dim, T=T, start="basis", reorth=True)
    lnZ = np.zeros(len(T))
    for i in range(3):
        si = oracle.System(two_s=[w["two_s"][i]], J=np.zeros((1, 1)), g=w["g"], B=w["B"],
                           d_ion=[w["d_ion"][i]], e_axes=[w["e_axes"][i]])
        ev = np.linalg.eigvalsh(dense.hamiltonian(si))
        for t, Tk in enumerate(T):
            lnZ[t] += np.log(np.sum(np.exp(-(ev - ev.min()) / Tk))) - ev.min() / Tk
    assert _rel(r["lnZ"], lnZ) < 1e-10


def test_breakdown_truncates_krylov_space():
    """A field along z only makes H diagonal: a basis vector is an eigenvector,
    Lanczos breaks down after one step (M_eff = 1) and the result is exact."""
    s = oracle.System(two_s=[1, 2], J=np.zeros((2, 2)), g=2.0, B=[0, 0, 0.5])
    r = oracle.ftlm(s, R=6, M=10, T=T, start="basis")
    assert list(r["M_eff"]) == [1] * 6
    ex = dense.thermo_exact(s, T)
    assert _rel(r["E"], ex["E"], 1e-6) < 1e-12


def test_sums_single_level():
    """One run, one Lanczos step: Z = d e^{-beta alpha}, E = alpha, C = 0, and
    the observable <r|O|r> = <O r|r> = conj(p_0), so M_B + i M_B_imag = -g conj(p_0)."""
    a = np.array([[1.5]]); b = np.array([[0.0]]); p = np.array([[0.25 + 0.1j]])
    r = oracle.ftlm_sums(a, b, p, [1], dim=8, g=2.0, T=T)
    assert np.allclose(r["lnZ"], np.log(8) - 1.5 / T)
    assert np.allclose(r["E"], 1.5) and np.allclose(r["C"], 0.0)
    assert np.allclose(r["M_B"], -0.5) and np.allclose(r["M_B_imag"], 0.2)


def test_random_vector_ftlm_converges_statistically():
    """Finite-R FTLM is statistical (parity unpinned at tolerance level); only
    a loose sanity bound: the N=6 s=1 ring, R = 10, M = 80 vs ED, T >= 1 K."""
    s = oracle_system(W.ring6_s1())
    r = oracle.ftlm(s, R=10, M=80, T=T, seed=0)
    ex = dense.thermo_exact(s, T)
    hi = T >= 1.0
    assert np.max(np.abs(r["E"][hi] - ex["E"][hi]) / np.abs(ex["E"][hi]).max()) < 0.1


def test_high_temperature_limits():
    """T -> infinity with every term of Eq. (3): E -> tr H / d =
    sum_i d_i s_i(s_i+1)/3 (exchange, dipolar and Zeeman terms are traceless),
    with E - tr H / d = -Var(H) / T + O(1/T^2); and the Curie law
    M_B T -> g^2 mu_B |B| sum_i s_i(s_i+1)/3, since to first order in beta
    <B^.S> = -beta tr((B^.S) H) / d and only the Zeeman term contributes."""
    w = random_system(np.random.default_rng(2607), [1, 2, 1, 3], scale=6.0)
    s = oracle_system(w)
    sv = np.asarray(w["two_s"]) / 2.0
    Tk = np.array([1e6, 1e7])
    r = oracle.ftlm(s, R=s.dim, M=s.dim, T=Tk, start="basis", reorth=True)
    e1 = np.sum(w["d_ion"] * sv * (sv + 1) / 3)
    dev = (r["E"] - e1) * Tk
    assert dev[0] < 0 and dev[1] < 0                      # -Var(H) < 0
    assert abs(dev[0] / dev[1] - 1) < 1e-3                 # the 1/T term
    assert np.all(np.abs(r["E"] - e1) < 1e-3 * max(1.0, abs(e1)))
    curie = w["g"] ** 2 * MU_B * np.linalg.norm(w["B"]) * np.sum(sv * (sv + 1) / 3)
    assert abs(r["M_B"][0] * Tk[0] / curie - 1) < 1e-4
    assert abs(r["M_B"][1] * Tk[1] / curie - 1) < 1e-5


def test_thermodynamics_invariant_under_rotation_and_field_reversal():
    """Rotating positions, axes and B together, or reversing B (time
    reversal), leaves ln Z, E, C and M_B unchanged: the oracle's FTLM in exact
    mode on the three systems (M_B is measured along B^ of each)."""
    rng = np.random.default_rng(7)
    w = random_system(rng, [1, 2, 1, 2])
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    Rm = q * np.sign(np.linalg.det(q))                    # a proper rotation
    variants = [w, dict(w, pos=w["pos"] @ Rm.T, e_axes=w["e_axes"] @ Rm.T, B=Rm @ w["B"]), dict(w, B=-w["B"])]
    res = []
    for v in variants:
        s = oracle_system(v)
        res.append(oracle.ftlm(s, R=s.dim, M=s.dim, T=T, start="basis", reorth=True))
    for r in res[1:]:
        for k in ("lnZ", "E", "C", "M_B"):
            assert _rel(r[k], res[0][k], 1e-6) < 1e-10, k
