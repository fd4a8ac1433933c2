"""Definition-level oracle: H as an explicit matrix -- TEST INFRASTRUCTURE ONLY.

Eq. (3) of the paper is written out literally with Kronecker products of the
spin matrices s^x, s^y, s^z of every site: no ladder expansion, no
hand-derived coefficients.  Exact diagonalisation (``numpy.linalg.eigh``)
then gives the thermal traces Tr(e^{-beta H}) and Tr(O e^{-beta H}) that the
FTLM estimators of Eqs. (4)-(5) approximate.  Intended for d up to a few
thousand.

Basis convention (shared reading, not shared code): index mu = sum_i a_i
prod_{k<i} q_k, site 0 least significant, digit a_i = m_i + s_i, so in a
Kronecker product site 0 is the rightmost factor.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def spin_matrices(two_s: int):
    """s^x, s^y, s^z for spin s = two_s / 2 in the basis a = m + s = 0..2s."""
    s = two_s / 2.0
    q = two_s + 1
    m = np.arange(q) - s
    sz = np.diag(m).astype(np.complex128)
    splus = np.zeros((q, q), dtype=np.complex128)
    for a in range(q - 1):  # s+ |m> = sqrt(s(s+1) - m(m+1)) |m+1>
        splus[a + 1, a] = np.sqrt(s * (s + 1) - m[a] * (m[a] + 1))
    sminus = splus.conj().T
    sx = (splus + sminus) / 2
    sy = (splus - sminus) / 2j
    return sx, sy, sz


def site_operators(two_s):
    """For every site i, the three embedded operators s_i^{x,y,z} (d x d,
    scipy.sparse CSR): I (x) ... (x) s^a (x) ... (x) I with site 0 rightmost."""
    two_s = list(two_s)
    n = len(two_s)
    dims = [t + 1 for t in two_s]
    ops = []
    for i in range(n):
        loc = spin_matrices(two_s[i])
        per = []
        for a in range(3):
            mat = sp.identity(1, dtype=np.complex128, format="csr")
            for k in reversed(range(n)):  # site n-1 leftmost, site 0 rightmost
                f = sp.csr_matrix(loc[a]) if k == i else sp.identity(dims[k], dtype=np.complex128, format="csr")
                mat = sp.kron(mat, f, format="csr")
            per.append(mat)
        ops.append(per)
    return ops


def hamiltonian_sparse(sys):
    """H of Eq. (3) for an ``oracle.System`` as a scipy.sparse matrix."""
    n = sys.n
    S = site_operators(sys.two_s)
    d = S[0][0].shape[0]
    H = sp.csr_matrix((d, d), dtype=np.complex128)
    for i in range(n):
        for j in range(i + 1, n):
            sisj = sum(S[i][a] @ S[j][a] for a in range(3))
            H += 2.0 * sys.J[i, j] * sisj
            if sys.pos is not None:
                rv = sys.pos[j] - sys.pos[i]
                r = np.linalg.norm(rv)
                e = rv / r
                si_e = sum(e[a] * S[i][a] for a in range(3))
                sj_e = sum(e[a] * S[j][a] for a in range(3))
                H += sys.C_dip * sys.g ** 2 / r ** 3 * (sisj - 3.0 * si_e @ sj_e)
    for i in range(n):
        if sys.d_ion is not None and sys.d_ion[i] != 0.0:
            e = sys.e_axes[i] / np.linalg.norm(sys.e_axes[i])
            se = sum(e[a] * S[i][a] for a in range(3))
            H += sys.d_ion[i] * se @ se
        H += sys.mu_B * sys.g * sum(sys.B[a] * S[i][a] for a in range(3))
    return H.tocsr()


def hamiltonian(sys) -> np.ndarray:
    """Dense H of Eq. (3) (for exact diagonalisation)."""
    return hamiltonian_sparse(sys).toarray()


def total_spin_along(sys, u) -> np.ndarray:
    S = site_operators(sys.two_s)
    u = np.asarray(u, dtype=np.float64)
    return sum(u[a] * S[i][a] for i in range(sys.n) for a in range(3)).toarray()


def field_direction(sys) -> np.ndarray:
    b = np.linalg.norm(sys.B)
    return sys.B / b if b > 0 else np.array([0.0, 0.0, 1.0])


def thermo_exact(sys, T, direction=None, H=None):
    """Exact lnZ, E, C, M_B (= -g <u.S>) by diagonalisation."""
    H = hamiltonian(sys) if H is None else H
    u = field_direction(sys) if direction is None else np.asarray(direction, dtype=np.float64)
    w, V = np.linalg.eigh(H)
    O = total_spin_along(sys, u)
    o_diag = np.real(np.einsum("ik,ij,jk->k", V.conj(), O, V))
    E0 = w.min()
    out = {k: np.empty(len(T)) for k in ("lnZ", "E", "C", "M_B")}
    for t, Tk in enumerate(T):
        b = 1.0 / Tk
        x = np.exp(-b * (w - E0))
        z = x.sum()
        Em = (x * w).sum() / z
        out["lnZ"][t] = np.log(z) - b * E0
        out["E"][t] = Em
        out["C"][t] = b * b * (x * (w - Em) ** 2).sum() / z
        out["M_B"][t] = -sys.g * (x * o_diag).sum() / z
    out["E0"] = E0
    return out


def thermo_from_vectors(sys, T, vecs, direction=None, H=None):
    """Exact stochastic-trace values for a fixed set of start vectors:
    Z = d/R sum_r <r|e^{-bH}|r>, O = sum_r <r|O e^{-bH}|r> / sum_r <r|e^{-bH}|r>
    (Eqs. 1, 4, 5 with the Krylov space complete).  vecs: [d][R], normalised."""
    H = hamiltonian(sys) if H is None else H
    u = field_direction(sys) if direction is None else np.asarray(direction, dtype=np.float64)
    w, V = np.linalg.eigh(H)
    O = total_spin_along(sys, u)
    d, R = vecs.shape
    c = V.conj().T @ vecs               # <k|r>
    Or = V.conj().T @ (O @ vecs)        # <k|O r> ;  <r|O|k> = conj(<k|O r>)
    E0 = w.min()
    out = {k: np.empty(len(T)) for k in ("lnZ", "E", "C", "M_B", "M_B_imag")}
    for t, Tk in enumerate(T):
        b = 1.0 / Tk
        x = np.exp(-b * (w - E0))
        wk = (np.abs(c) ** 2 * x[:, None]).sum(axis=1)   # weight per eigenstate
        z = wk.sum()
        Em = (wk * w).sum() / z
        o = (np.conj(Or) * x[:, None] * c).sum()
        out["lnZ"][t] = np.log(d / R * z) - b * E0
        out["E"][t] = Em
        out["C"][t] = b * b * (wk * (w - Em) ** 2).sum() / z
        out["M_B"][t] = -sys.g * np.real(o) / z
        out["M_B_imag"][t] = -sys.g * np.imag(o) / z
    return out


def time_reversal_unitary(two_s):
    """U = (x)_i exp(-i pi s^y_i) (site 0 rightmost), so that the time-reversal
    operator is Theta x = U conj(x) (Sec. II.B).  Built with scipy's expm of
    each site's s^y matrix, independently of any closed form."""
    import scipy.linalg as sla
    U = np.ones((1, 1), dtype=np.complex128)
    for t in reversed(list(two_s)):  # site n-1 leftmost
        U = np.kron(U, sla.expm(-1j * np.pi * spin_matrices(t)[1]))
    return U
