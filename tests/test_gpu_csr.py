"""The stored-matrix comparison path (Sec. II.C, Table I: the matrix kept on
the GPU, one thread per row): assembled on the device from the same row
enumeration as the matrix-free gather, checked element count and products
against the FP64 oracle.  Tolerances as the matvec tests."""
import numpy as np
import pytest
from conftest import random_system
from gpu_helpers import empty_dev, osys, rel_l2, sampled_rows_reference, to_dev, torch_cuda

import ftlm_workloads as W
import oracle
import paper_2607_25585_gb300 as F

pytestmark = pytest.mark.gpu
TOL = {"c128": 1e-12, "c64": 2e-5}

SYSTEMS = {
    "mixed_spins": lambda rng: random_system(rng, [1, 2, 3, 5, 1, 2]),
    "ring6_s1": lambda rng: W.ring6_s1(),
    "lattice4x3": lambda rng: W.square_lattice(4, 3, seed=1),
    "spin52_pair": lambda rng: random_system(rng, [5, 5, 4]),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    F.build()
    torch_cuda()


@pytest.mark.parametrize("name", sorted(SYSTEMS))
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_csr_matches_oracle(name, dtype, rng):
    w = SYSTEMS[name](rng)
    s = F.System.from_dict(w)
    m = F.CsrMatrix(s, dtype)
    os_ = osys(w)
    # element count: every nonzero element of H (the oracle's columns; H is Hermitian)
    nz = 0
    for nu in range(s.dim):
        _, v = oracle.h_column(os_, nu)
        nz += int(np.count_nonzero(np.abs(v) > 1e-13))
    assert m.nnz == nz
    for R in (1, 3, 64):
        x = rng.normal(size=(s.dim, R)) + 1j * rng.normal(size=(s.dim, R))
        if dtype == "c64":
            x = x.astype(np.complex64).astype(np.complex128)
        y = empty_dev((s.dim, R), dtype)
        m.apply(to_dev(x, dtype), y, R)
        assert rel_l2(y.cpu().numpy(), oracle.apply_h(os_, x)) < TOL[dtype]
    m.close()


def test_csr_full_size_sampled_rows(rng):
    """d = 1,048,576 (2.2e8 stored elements) x R = 64 complex64: sampled rows."""
    w = W.lattice4x5()
    s = F.System.from_dict(w)
    m = F.CsrMatrix(s, "c64")
    assert m.nnz == s.dim * (1 + 20 + 190)  # all-pairs dipolar: every pair and site flip present
    torch = torch_cuda()
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randn(s.dim, 64, dtype=torch.complex64, device="cuda", generator=g)
    y = torch.empty_like(x)
    m.apply(x, y, 64)
    rows = np.unique(np.concatenate([[0, s.dim - 1], rng.integers(0, s.dim, size=10)]))
    ref = sampled_rows_reference(w, x, rows)
    assert rel_l2(y[torch.from_numpy(rows).cuda()].cpu().numpy(), ref) < TOL["c64"]
    m.close()


def test_csr_rejects_bad_blocks():
    s = F.System.from_dict(W.square_lattice(2, 2, seed=1))
    m = F.CsrMatrix(s, "c64")
    torch = torch_cuda()
    x = torch.zeros(s.dim, 4, dtype=torch.complex64, device="cuda")
    with pytest.raises(F.FtlmError):
        m.apply(x, x, 4)
    with pytest.raises(F.FtlmError):
        m.apply(x, torch.zeros_like(x), 0)
    m.close()
