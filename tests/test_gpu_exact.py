"""The GPU path in the exact limits of FTLM, against exact diagonalisation
(LAPACK on the dense Hamiltonian of Eq. 3), and the optional full
re-orthogonalisation of Sec. II.C against the oracle.

With every basis vector as a start vector and the Krylov space complete
(M = d), Eqs. (4)-(5) are the exact traces Tr(e^{-H/T}), Tr(H e^{-H/T}) and
Tr(u.S e^{-H/T}), so ln Z, E, C and M_B equal exact diagonalisation up to
rounding: 1e-10 relative in complex128 (the oracle's own exact mode meets
the same bound at d <= 729)."""
import numpy as np
import pytest
from gpu_helpers import osys, torch_cuda

import ftlm_workloads as W
import oracle
import paper_2607_25585_gb300 as F
from oracle import dense

pytestmark = pytest.mark.gpu
T = W.temperatures()
KEYS = ("lnZ", "E", "C", "M_B")


@pytest.fixture(scope="module", autouse=True)
def built():
    F.build()
    torch_cuda()


def rel(a, b, floor=1e-6, mask=None):
    a, b = np.asarray(a), np.asarray(b)
    if mask is not None:
        a, b = a[mask], b[mask]
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor * np.max(np.abs(b)))))


def exact_mode(s, dtype, chunk, reorth=False):
    """FTLM on all basis vectors, M = d, in runs of `chunk` vectors merged on
    the host by ftlm_sums (the multi-process merge)."""
    d = s.dim
    parts = [F.run(s, R=min(chunk, d - off), M=d, T=T, start="basis", basis_offset=off, dtype=dtype, reorth=reorth)
             for off in range(0, d, chunk)]
    cat = {k: np.concatenate([p[k] for p in parts]) for k in ("alpha", "beta", "p", "M_eff")}
    return F.sums(cat["alpha"], cat["beta"], cat["p"], cat["M_eff"], d, s.g, T), cat


def test_ring6_exact_mode_equals_ed():
    """The N = 6, s = 1 ring (d = 729: tilted single-ion axes, field along
    (1,1,1), all-pairs dipolar coupling) on the hot path's recurrence (no
    re-orthogonalisation): all 729 basis vectors in three runs of 243, 729
    steps each.  complex128 within 1e-10 of exact diagonalisation; complex64
    (FP32 matvec, FP64 scalars) within 1e-4 for T >= 0.1 K."""
    w = W.ring6_s1()
    s = F.System.from_dict(w)
    ex = dense.thermo_exact(osys(w), T)
    r, cat = exact_mode(s, "c128", 243)
    assert np.all(cat["M_eff"] == s.dim)
    for k in KEYS:
        assert rel(r[k], ex[k]) < 1e-10, k
    r64, _ = exact_mode(s, "c64", 243)
    for k in KEYS:
        assert rel(r64[k], ex[k], 1e-3, T >= 0.1) < 1e-4, k


def test_reorth_matches_oracle():
    """Full re-orthogonalisation (reorth = 1) against the oracle's, same
    Philox vectors, on the N = 5 s = 1 ring (d = 243) with 100 steps (past the
    first Ritz convergence, where the plain recurrence of the two would
    drift apart): alpha, beta, p over all steps and the thermodynamics to
    1e-10 in complex128."""
    w = W.ring(N=5, two_s=2)
    s = F.System.from_dict(w)
    R, M = 4, 100
    g = F.run(s, R=R, M=M, T=T, seed=3, dtype="c128", reorth=True)
    o = oracle.ftlm(osys(w), R=R, M=M, T=T, seed=3, reorth=True)
    assert list(g["M_eff"]) == list(o["M_eff"])
    for r in range(R):
        m = o["M_eff"][r]
        sa = np.abs(o["alpha"][r, :m]).max()
        assert np.max(np.abs(g["alpha"][r, :m] - o["alpha"][r, :m])) < 1e-10 * sa
        assert np.max(np.abs(g["beta"][r, : m - 1] - o["beta"][r, : m - 1])) < 1e-10 * sa
        assert np.max(np.abs(g["p"][r, :m] - o["p"][r, :m])) < 1e-10 * max(1.0, np.abs(o["p"][r, :m]).max())
    for k in KEYS:
        assert rel(g[k], o[k], 1e-3, T >= 0.1) < 1e-10, k


def test_reorth_exact_mode_equals_ed():
    """Exact mode with full re-orthogonalisation on the N = 4 s = 1 ring
    (d = 81, all basis vectors, M = d): complex128 within 1e-10 of exact
    diagonalisation, complex64 within 1e-4 (T >= 0.1 K)."""
    w = W.ring(N=4, two_s=2)
    s = F.System.from_dict(w)
    ex = dense.thermo_exact(osys(w), T)
    r, _ = exact_mode(s, "c128", 81, reorth=True)
    for k in KEYS:
        assert rel(r[k], ex[k]) < 1e-10, k
    r64, _ = exact_mode(s, "c64", 81, reorth=True)
    for k in KEYS:
        assert rel(r64[k], ex[k], 1e-3, T >= 0.1) < 1e-4, k


def test_reorth_refused_for_batches():
    systems = [F.System.from_dict(W.chain(N, two_s=2)) for N in (4, 5)]
    with pytest.raises(F.FtlmError, match="UNSUPPORTED"):
        F.run_batch(systems, R=2, M=5, T=T, dtype="c128", reorth=True)
