"""GPU parity of symmetric FTLM (Eqs. E-2-G, E-2-H): the stored Lanczos
vectors, the matrix O_ij = <v_i|u.S|v_j> formed on the device (u.S on the
stored vectors, then their contraction with the stored vectors) and the host double sum, against the
FP64 oracle with the same random vectors.  complex128: O over the first 15
steps to 1e-10 (before the Lanczos runs part by finite precision) and M_B_sym
to 1e-9 for T >= 0.1 K; complex64: M_B_sym to 1e-4."""
import numpy as np
import pytest
from conftest import random_system
from gpu_helpers import osys, torch_cuda

import ftlm_workloads as W
import oracle
import paper_2607_25585_gb300 as F

pytestmark = pytest.mark.gpu
T = W.temperatures()


@pytest.fixture(scope="module", autouse=True)
def built():
    F.build()
    torch_cuda()


def rel(a, b, floor=1e-3, mask=None):
    a, b = np.asarray(a), np.asarray(b)
    if mask is not None:
        a, b = a[mask], b[mask]
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor * np.max(np.abs(b)))))


CASES = {
    "lattice4x3": lambda rng: (W.square_lattice(4, 3, seed=1), "random"),   # vector-major gather
    "mixed": lambda rng: (random_system(rng, [1, 2, 3, 1, 2]), "pairs"),    # general kernel, row-major
    "mn9_small": lambda rng: (W.mn9(vertices=3, Bdir=W.dodecahedron_directions()[2]), "pairs"),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_sftlm_matches_oracle(name, rng):
    w, start = CASES[name](rng)
    s = F.System.from_dict(w)
    o = oracle.sftlm(osys(w), R=4, M=30, T=T, seed=8, start=start)
    g = F.run(s, R=4, M=30, T=T, seed=8, start=start, dtype="c128", symmetric=True)
    cold = T >= 0.1
    for k in ("lnZ", "E", "C", "M_B"):
        assert rel(g[k], o[k], 1e-3, cold) < 1e-9, k
    assert rel(g["M_B_sym"], o["M_B_sym"], 1e-3, cold) < 1e-9
    for r in range(4):
        m = min(15, o["M_eff"][r])
        so = np.abs(o["O"][r, :m, :m]).max()
        assert np.max(np.abs(g["O"][r, :m, :m] - o["O"][r, :m, :m])) < 1e-10 * so
    assert g["sym_ms"] > 0
    g64 = F.run(s, R=4, M=30, T=T, seed=8, start=start, dtype="c64", symmetric=True)
    assert rel(g64["M_B_sym"], o["M_B_sym"], 1e-3, cold) < 1e-4


def test_sftlm_reuses_plain_run_results(rng):
    """A symmetric run returns the same FTLM outputs as a plain run (the
    extra copies do not change the recurrence)."""
    w = W.square_lattice(4, 3, seed=2)
    s = F.System.from_dict(w)
    a = F.run(s, R=6, M=25, T=T, seed=1, dtype="c64")
    b = F.run(s, R=6, M=25, T=T, seed=1, dtype="c64", symmetric=True)
    for k in ("alpha", "beta", "p"):
        assert np.array_equal(a[k], b[k])


def test_symmetric_batch_rejected():
    ws = [W.square_lattice(2, 2, seed=1), W.square_lattice(2, 3, seed=1)]
    systems = [F.System.from_dict(w) for w in ws]
    keep = []
    p = F._params(2, 5, T, 0, 0, "c64", "random", 0, None, None, 0.0, False, False, None, keep, True)
    import ctypes
    rs = (F.Result * 2)()
    handles = (ctypes.c_void_p * 2)(*[x.handle for x in systems])
    assert F.lib().ftlm_run_batch(2, handles, ctypes.byref(p), rs) != 0


@pytest.mark.parametrize("M", [8, 40, 70])
def test_sftlm_block_sizes(M):
    """The contraction's blocks of 16, 48 and 64 vectors (T = 1, 3, 4 entries a
    thread per side; M = 70 spans two blocks per side): O over the first
    steps against the oracle (complex128, 1e-10), and every entry of O
    against its Hermitian partner, which the kernel forms from other tiles
    and, for M = 70, in another CTA."""
    w = W.square_lattice(4, 3, seed=3)
    s = F.System.from_dict(w)
    R = 2
    o = oracle.sftlm(osys(w), R=R, M=M, T=T, seed=4)
    g = F.run(s, R=R, M=M, T=T, seed=4, dtype="c128", symmetric=True)
    for r in range(R):
        me = int(g["M_eff"][r])
        assert me == M
        O = g["O"][r, :me, :me]
        so = np.abs(O).max()
        assert np.max(np.abs(O - O.conj().T)) < 1e-12 * so
        m = min(8, me)
        assert np.max(np.abs(O[:m, :m] - o["O"][r, :m, :m])) < 1e-10 * so
        if M > 64:  # entries of the second block row and column
            assert np.abs(O[64:, :]).max() > 1e-3 * so and np.abs(O[:, 64:]).max() > 1e-3 * so
    s.close()
