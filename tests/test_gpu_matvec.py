"""GPU parity of the matrix-free H.v (Eq. 3), the observable u.S and the
random start block against the FP64 oracle, through the C ABI.

Tolerances: complex128 to 1e-12 relative L2 (the FP64 path evaluates the
same sums in another order).  complex64: every output row is a sum of K
terms rounded in FP32 (unit roundoff u = 2^-24 ~ 6e-8); the accumulated
error is bounded by ~K u sum|terms| and behaves like sqrt(K) u in practice.
With K <= ~400 terms per row for these systems and cancellation between terms
of both signs, the test bound is 2e-5 relative L2 on random inputs."""
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
    "mixed_spins": lambda rng: random_system(rng, [1, 2, 3, 5, 1, 2]),   # d = 864, every term
    "ring6_s1": lambda rng: W.ring6_s1(),                                  # d = 729
    "lattice4x3": lambda rng: W.square_lattice(4, 3, seed=1),              # d = 4096 s = 1/2
    "chain7_s1": lambda rng: W.chain(7, Bdir=(0.3, -0.2, 0.9)),            # d = 2187
    "spin52_pair": lambda rng: random_system(rng, [5, 5, 4]),              # s = 5/2, 2: +-2 steps
}


@pytest.fixture(scope="module", autouse=True)
def built():
    F.build()
    torch_cuda()


@pytest.mark.parametrize("name", sorted(SYSTEMS))
@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("R", [1, 3, 4, 8, 10, 64])
def test_apply_h_matches_oracle(name, dtype, R, rng):
    w = SYSTEMS[name](rng)
    s = F.System.from_dict(w)
    d = s.dim
    x = rng.normal(size=(d, R)) + 1j * rng.normal(size=(d, R))
    if dtype == "c64":
        x = x.astype(np.complex64).astype(np.complex128)  # the oracle sees the same rounded input
    ref = oracle.apply_h(osys(w), x)
    xd = to_dev(x, dtype)
    yd = empty_dev((d, R), dtype)
    F.apply_h(s, xd, yd, R, dtype)
    y = yd.cpu().numpy()
    assert rel_l2(y, ref) < TOL[dtype]


@pytest.mark.parametrize("name", sorted(SYSTEMS))
def test_apply_h_c64_per_row_bound(name, rng):
    """complex64, row by row: |y_mu - (Hx)_mu| <= 1e-5 * sum_nu |H_mu,nu| |x_nu|.
    The bound is what FP32 products and sums can lose (coefficients rounded
    to FP32, ~K u relative to the sum of absolute terms for K terms), so a
    wrong or missing term in any single row fails it even when the block-wide
    relative L2 would hide it."""
    from oracle import dense
    w = SYSTEMS[name](rng)
    s = F.System.from_dict(w)
    d, R = s.dim, 8
    x = rng.normal(size=(d, R)) + 1j * rng.normal(size=(d, R))
    x = x.astype(np.complex64).astype(np.complex128)
    H = dense.hamiltonian(osys(w))
    ref = H @ x
    bound = np.abs(H) @ np.abs(x)
    yd = empty_dev((d, R), "c64")
    F.apply_h(s, to_dev(x, "c64"), yd, R, "c64")
    err = np.abs(yd.cpu().numpy() - ref)
    assert np.all(bound > 0)
    assert np.max(err / bound) < 1e-5


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("shape", [(0, 1, 2), (2, 1, 1), (2, 5, 4), (3, 10, 2), (4, 2, 1), (4, 10, 8), (3, 3, 2),
                                   (2, 1, 1, 1), (3, 10, 2, 1), (3, 3, 4, 1), (4, 5, 4, 1), (4, 10, 8, 1),
                                   (3, 1, 1, 3), (4, 1, 2, 4)])
def test_apply_h_every_kernel_variant(dtype, shape, rng):
    """General kernel (cube_bits 0) and the spin-1/2 register-cube kernel
    with every cube size, several vector-group widths (incl. groups that do
    not divide R) and tile sizes, in one pass or in ceil(N/K) passes (the
    4x4 lattice with K = 3 has an overlapping last cube),
    on 4x3 and 4x4 lattices.  The vector-major shapes (multipass 3, 4) fall
    back to the row-major cube kernel for row-major blocks."""
    for w in (W.square_lattice(4, 3, seed=1), W.square_lattice(4, 4, seed=2)):
        s = F.System.from_dict(w)
        d, R = s.dim, 10
        x = rng.normal(size=(d, R)) + 1j * rng.normal(size=(d, R))
        if dtype == "c64":
            x = x.astype(np.complex64).astype(np.complex128)
        ref = oracle.apply_h(osys(w), x)
        try:
            F.tune_shape(s, R, dtype, *shape)
            yd = empty_dev((d, R), dtype)
            F.apply_h(s, to_dev(x, dtype), yd, R, dtype)
            assert rel_l2(yd.cpu().numpy(), ref) < TOL[dtype]
        finally:
            F.tune_shape(s, R, dtype, -1)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_apply_sdir_matches_oracle(dtype, rng):
    w = random_system(rng, [2, 1, 3, 2])
    s = F.System.from_dict(w)
    d, R = s.dim, 4
    x = rng.normal(size=(d, R)) + 1j * rng.normal(size=(d, R))
    if dtype == "c64":
        x = x.astype(np.complex64).astype(np.complex128)
    for u in (None, np.array([0.3, -0.5, 0.8])):
        uu = w["B"] / np.linalg.norm(w["B"]) if u is None else u / np.linalg.norm(u)
        ref = oracle.apply_sdir(osys(w), uu, x)
        yd = empty_dev((d, R), dtype)
        F.apply_sdir(s, to_dev(x, dtype), yd, R, dtype, u=u)
        assert rel_l2(yd.cpu().numpy(), ref) < TOL[dtype]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_start_block_matches_oracle(dtype):
    w = W.square_lattice(4, 3, seed=1)
    s = F.System.from_dict(w)
    d = s.dim
    for R, off in ((5, 0), (3, 7), (64, 0)):
        ref = oracle.start_vectors(d, R, seed=42, vec_offset=off)
        out = empty_dev((d, R), dtype)
        F.start_block(s, out, R, seed=42, vec_offset=off, dtype=dtype)
        got = out.cpu().numpy()
        assert rel_l2(got, ref) < (1e-14 if dtype == "c128" else 1e-7)
        assert np.allclose(np.linalg.norm(got, axis=0), 1.0, atol=1e-6 if dtype == "c64" else 1e-14)


def test_apply_h_bitwise_deterministic(rng):
    w = W.square_lattice(4, 4, seed=1)
    s = F.System.from_dict(w)
    d, R = s.dim, 64
    torch = torch_cuda()
    x = torch.randn(d, R, dtype=torch.complex64, device="cuda")
    y1 = torch.empty_like(x)
    y2 = torch.empty_like(x)
    F.apply_h(s, x, y1, R, "c64")
    F.apply_h(s, x, y2, R, "c64")
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)


def test_apply_h_rejects_bad_blocks():
    s = F.System.from_dict(W.square_lattice(2, 2, seed=1))
    torch = torch_cuda()
    x = torch.zeros(s.dim, 4, dtype=torch.complex64, device="cuda")
    with pytest.raises(F.FtlmError):
        F.apply_h(s, x, x, 4, "c64")              # overlapping
    with pytest.raises(F.FtlmError):
        F.apply_h(s, x, torch.zeros_like(x), 0, "c64")
    with pytest.raises(F.FtlmError):
        F.apply_h(s, x, torch.zeros_like(x), 1024, "c64")


# ---- full size, in the launch configuration the benchmark times --------------

@pytest.mark.parametrize("wname,R", [("lattice4x5", 64), ("lattice4x4", 50)])
def test_full_size_sampled_rows(wname, R, rng):
    """d = 1,048,576 x R = 64 (complex64) and d = 65,536 x R = 50: sampled
    output rows, including the first and last (ragged tail), against the
    oracle evaluated row by row."""
    w = W.WORKLOADS[wname]["system"]()
    s = F.System.from_dict(w)
    d = s.dim
    torch = torch_cuda()
    g = torch.Generator(device="cuda").manual_seed(7)
    x = torch.randn(d, R, dtype=torch.complex64, device="cuda", generator=g)
    y = torch.empty_like(x)
    F.apply_h(s, x, y, R, "c64")
    rows = np.unique(np.concatenate([[0, d - 1, d // 2], rng.integers(0, d, size=12)]))
    ref = sampled_rows_reference(w, x, rows)
    got = y[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert rel_l2(got, ref) < TOL["c64"]


def test_full_size_hermitian(rng):
    """<x|H y> = conj(<y|H x>) at d = 1,048,576 with all-pairs dipolar terms."""
    w = W.lattice4x5()
    s = F.System.from_dict(w)
    d = s.dim
    torch = torch_cuda()
    x = torch.randn(d, 2, dtype=torch.complex64, device="cuda")
    hx = torch.empty_like(x)
    F.apply_h(s, x, hx, 2, "c64")
    a = torch.vdot(x[:, 0].to(torch.complex128), hx[:, 1].to(torch.complex128)).item()
    b = torch.vdot(x[:, 1].to(torch.complex128), hx[:, 0].to(torch.complex128)).item()
    assert abs(a - np.conj(b)) < 1e-5 * abs(a)


def test_ladder_sampled_rows(rng):
    """d = 67,108,864 (2 x 13 ladder) x R = 4, complex64: sampled rows."""
    w = W.ladder2x13()
    s = F.System.from_dict(w)
    d, R = s.dim, 4
    torch = torch_cuda()
    x = torch.randn(d, R, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    F.apply_h(s, x, y, R, "c64")
    rows = np.unique(np.concatenate([[0, d - 1], rng.integers(0, d, size=6)]))
    ref = sampled_rows_reference(w, x, rows)
    got = y[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert rel_l2(got, ref) < TOL["c64"]
    del x, y
