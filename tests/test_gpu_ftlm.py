"""GPU parity of the whole FTLM path (start block, Lanczos recurrence with
fused reductions, host eigensolve, sums of Eqs. 4-5) against the FP64
oracle with the identical Philox random vectors, through the C ABI.

complex128: the same algorithm in FP64.  alpha, beta, p agree to 1e-10
relative over the steps before the first Ritz value converges (here the
first 20; measured first divergence 36-72 steps).  Later, Lanczos without
re-orthogonalisation amplifies rounding-order differences (ghost Ritz
values), so two correct FP64 runs no longer agree step by step.  The
Gauss-quadrature sums stay stable, and lnZ, E, C, M_B agree to 1e-10 for
T >= 0.1 K at full depth (measured <= 3e-11).  complex64 (FP32 matvec, FP64
scalars): lnZ, E, C, M_B within 1e-4 relative of the FP64 oracle for
T >= 0.1 K (measured <= 2.4e-5).  Quantities passing through zero get a
floor of 1e-3 of their maximum over T."""
import numpy as np
import pytest
from conftest import random_system
from gpu_helpers import osys, to_dev, torch_cuda

import ftlm_workloads as W
import oracle
import paper_2607_25585_gb300 as F

pytestmark = pytest.mark.gpu
T = W.temperatures()
KEYS = ("lnZ", "E", "C", "M_B")


@pytest.fixture(scope="module", autouse=True)
def built():
    F.build()
    torch_cuda()


def rel(a, b, floor=1e-3, mask=None):
    a, b = np.asarray(a), np.asarray(b)
    if mask is not None:
        a, b = a[mask], b[mask]
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor * np.max(np.abs(b)))))


def compare_tridiag(g, o, tol, steps=20):
    R = o["alpha"].shape[0]
    assert list(g["M_eff"]) == list(o["M_eff"])
    for r in range(R):
        m = min(o["M_eff"][r], steps)
        sa = np.abs(o["alpha"][r, :m]).max()
        assert np.max(np.abs(g["alpha"][r, :m] - o["alpha"][r, :m])) < tol * sa
        assert np.max(np.abs(g["beta"][r, : m - 1] - o["beta"][r, : m - 1])) < tol * sa
        assert np.max(np.abs(g["p"][r, :m] - o["p"][r, :m])) < tol * max(1.0, np.abs(o["p"][r, :m]).max())


@pytest.mark.parametrize("case", ["ring6_s1", "mixed", "lattice4x3"])
def test_ftlm_c128_matches_oracle(case):
    if case == "ring6_s1":
        w, R, M = W.ring6_s1(), 10, 80
    elif case == "mixed":  # its own generator: the system must not depend on the order tests run in
        w, R, M = random_system(np.random.default_rng(2607), [1, 2, 3, 2]), 5, 40
    else:
        w, R, M = W.square_lattice(4, 3, seed=1), 6, 60
    s = F.System.from_dict(w)
    g = F.run(s, R=R, M=M, T=T, seed=5, dtype="c128")
    o = oracle.ftlm(osys(w), R=R, M=M, T=T, seed=5)
    compare_tridiag(g, o, 1e-10)
    cold = T >= 0.1
    for k in KEYS:  # relative error with the module's floor for quantities passing through zero
        assert rel(g[k], o[k], 1e-3, cold) < 1e-10, k
        assert rel(g[k], o[k], 1e-3) < 1e-9, k
    assert abs(g["E0"] - o["E0"]) < 1e-10 * abs(o["E0"])


@pytest.mark.parametrize("case", ["ring6_s1", "lattice4x3"])
def test_ftlm_c64_within_1e4_of_fp64_oracle(case):
    w, R, M = (W.ring6_s1(), 10, 80) if case == "ring6_s1" else (W.square_lattice(4, 3, seed=1), 8, 60)
    s = F.System.from_dict(w)
    g = F.run(s, R=R, M=M, T=T, seed=0, dtype="c64")
    o = oracle.ftlm(osys(w), R=R, M=M, T=T, seed=0)
    cold = T >= 0.1
    for k in KEYS:
        assert rel(g[k], o[k], 1e-3, cold) < 1e-4, k


def test_ftlm_vec_offset_shards_vectors():
    """Vectors vec_offset .. vec_offset+R-1 of the same stream: two shards of
    3 reproduce the tridiagonal data of one run of 6."""
    w = W.ring(N=5, two_s=2)
    s = F.System.from_dict(w)
    full = F.run(s, R=6, M=30, T=T, seed=9, dtype="c128")
    a = F.run(s, R=3, M=30, T=T, seed=9, vec_offset=0, dtype="c128")
    b = F.run(s, R=3, M=30, T=T, seed=9, vec_offset=3, dtype="c128")
    for k in ("alpha", "beta", "p"):  # the pre-convergence steps (different block widths sum in another order)
        assert np.allclose(np.concatenate([a[k], b[k]])[:, :10], full[k][:, :10], rtol=1e-11, atol=1e-12)
    merged = F.sums(np.concatenate([a["alpha"], b["alpha"]]), np.concatenate([a["beta"], b["beta"]]),
                    np.concatenate([a["p"], b["p"]]), np.concatenate([a["M_eff"], b["M_eff"]]), s.dim, s.g, T)
    for k in KEYS:
        assert rel(merged[k], full[k], 1e-6, T >= 0.1) < 1e-10


def test_ftlm_basis_and_user_start(rng):
    w = random_system(rng, [1, 2, 1, 2])
    s = F.System.from_dict(w)
    d = s.dim
    g = F.run(s, R=4, M=12, T=T, start="basis", basis_offset=5, dtype="c128")
    o = oracle.ftlm(osys(w), R=4, M=12, T=T, start="basis", basis_offset=5)
    compare_tridiag(g, o, 1e-10)
    us = rng.normal(size=(d, 3)) + 1j * rng.normal(size=(d, 3))
    g = F.run(s, R=3, M=12, T=T, start="user", user_start=to_dev(us, "c128"), dtype="c128")
    o = oracle.ftlm(osys(w), R=3, M=12, T=T, start="user", user_start=us)
    compare_tridiag(g, o, 1e-10)
    for k in KEYS:
        assert rel(g[k], o[k], 1e-6, T >= 0.1) < 1e-10


def test_ftlm_observable_direction(rng):
    w = random_system(rng, [2, 1, 2])
    s = F.System.from_dict(w)
    u = np.array([0.2, 0.9, -0.3])
    g = F.run(s, R=3, M=15, T=T, seed=2, dtype="c128", obs_dir=u)
    o = oracle.ftlm(osys(w), R=3, M=15, T=T, seed=2, direction=u / np.linalg.norm(u))
    assert rel(g["M_B"], o["M_B"], 1e-6, T >= 0.1) < 1e-10


def test_ftlm_breakdown():
    """Diagonal H (field along z, no couplings): every basis vector is an
    eigenvector; the recurrence stops after one step."""
    s = F.System([1, 2], J=np.zeros((2, 2)), B=[0, 0, 0.5])
    for dt in ("c128", "c64"):
        g = F.run(s, R=6, M=10, T=T, start="basis", dtype=dt)
        assert list(g["M_eff"]) == [1] * 6
    o = oracle.ftlm(oracle.System(two_s=[1, 2], J=np.zeros((2, 2)), B=[0, 0, 0.5]), R=6, M=10, T=T, start="basis")
    assert rel(g["E"], o["E"], 1e-6) < 1e-6


def test_ftlm_batch_matches_single_runs():
    """Uneven-size instances in one graph reproduce their single runs."""
    ws = [W.chain(N, Bdir=bd, two_s=2) for N in (5, 6, 7) for bd in W.fibonacci_directions(2)]
    systems = [F.System.from_dict(w) for w in ws]
    outs = F.run_batch(systems, R=4, M=25, T=T, seed=3, dtype="c128")
    cold = T >= 0.1
    for w, s, b in zip(ws, systems, outs):
        single = F.run(s, R=4, M=25, T=T, seed=3, dtype="c128")
        o = oracle.ftlm(osys(w), R=4, M=25, T=T, seed=3)
        for k in KEYS:
            assert rel(b[k], single[k], 1e-6, cold) < 1e-10, k
            assert rel(b[k], o[k], 1e-6, cold) < 1e-10, k
    outs64 = F.run_batch(systems, R=4, M=25, T=T, seed=3, dtype="c64")
    for w, b in zip(ws, outs64):
        o = oracle.ftlm(osys(w), R=4, M=25, T=T, seed=3)
        for k in KEYS:
            assert rel(b[k], o[k], 1e-3, T >= 0.1) < 1e-4, k


def test_ftlm_bitwise_reproducible_and_timed():
    s = F.System.from_dict(W.square_lattice(4, 3, seed=1))
    a = F.run(s, R=8, M=20, T=T, seed=1, dtype="c64", time_kernels=True)
    b = F.run(s, R=8, M=20, T=T, seed=1, dtype="c64", time_kernels=True)
    for k in ("alpha", "beta", "p"):
        assert np.array_equal(a[k], b[k])
    assert a["hv_launches"] == 20 and a["hv_ms"] > 0 and a["device_ms"] >= a["hv_ms"]
    assert a["kernel_launches"] >= 2 * 20


def test_ftlm_autotune_same_answer():
    s = F.System.from_dict(W.square_lattice(4, 3, seed=1))
    a = F.run(s, R=8, M=20, T=T, seed=1, dtype="c128")
    b = F.run(s, R=8, M=20, T=T, seed=1, dtype="c128", autotune=True)
    for k in KEYS:  # another launch shape may sum in another order
        assert rel(a[k], b[k], 1e-6, T >= 0.1) < 1e-10


@pytest.mark.parametrize("shape", [(0, 1, 2), (2, 4, 1), (3, 8, 2), (4, 2, 4), (3, 8, 2, 1), (4, 8, 4, 1)])
def test_ftlm_every_kernel_variant(shape):
    """The spin-1/2 register-cube kernel (cube_bits 2..4, vector groups,
    tile sizes) and the general kernel give the oracle's FTLM."""
    w = W.square_lattice(4, 3, seed=1)
    s = F.System.from_dict(w)
    o = oracle.ftlm(osys(w), R=8, M=40, T=T, seed=6)
    try:
        for dt in ("c128", "c64"):
            F.tune_shape(s, 8, dt, *shape)
            g = F.run(s, R=8, M=40, T=T, seed=6, dtype=dt)
            tol = 1e-10 if dt == "c128" else 1e-4
            for k in KEYS:
                assert rel(g[k], o[k], 1e-3, T >= 0.1) < tol, (dt, k)
    finally:
        for dt in ("c128", "c64"):
            F.tune_shape(s, 8, dt, -1)


@pytest.mark.parametrize("shape", [(3, 1, 1, 3), (4, 1, 2, 3), (3, 1, 4, 4), (4, 1, 1, 4), (3, 1, 1, 5), (4, 1, 2, 5),
                                   (4, 1, 1, 6), (3, 1, 2, 7), (3, 1, 1, 8), (3, 1, 2, 9)])
def test_ftlm_vector_major_matches_oracle(shape, rng):
    """Vector-major Lanczos block (each vector contiguous; a warp owns 32
    consecutive rows, a thread a cube above them), in one pass, in passes
    whose cubes cover bits [5, n) (the last cube overlapping the one before),
    or in two passes (cubes on bits [5, 5+K) and on the top K bits):
    random start with a vector offset, basis start and a user block
    (transposed on the device) against the oracle step by step (complex128)
    and in the thermodynamics (complex64), on 4x3 and 4x4 lattices."""
    for w in (W.square_lattice(4, 3, seed=1), W.square_lattice(4, 4, seed=2)):
        s = F.System.from_dict(w)
        d = s.dim
        try:
            for R in (6, 3):
                for dt in ("c128", "c64"):
                    F.tune_shape(s, R, dt, *shape)
            g = F.run(s, R=6, M=30, T=T, seed=4, vec_offset=3, dtype="c128")
            assert g["shape"]["vector_major"] == 1
            o = oracle.ftlm(osys(w), R=6, M=30, T=T, seed=4, vec_offset=3)
            compare_tridiag(g, o, 1e-10)
            g64 = F.run(s, R=6, M=30, T=T, seed=4, vec_offset=3, dtype="c64")
            assert g64["shape"]["vector_major"] == 1
            for k in KEYS:
                assert rel(g64[k], o[k], 1e-3, T >= 0.1) < 1e-4, k
            g = F.run(s, R=3, M=12, T=T, start="basis", basis_offset=d - 3, dtype="c128")
            ob = oracle.ftlm(osys(w), R=3, M=12, T=T, start="basis", basis_offset=d - 3)
            compare_tridiag(g, ob, 1e-10)
            us = rng.normal(size=(d, 3)) + 1j * rng.normal(size=(d, 3))
            g = F.run(s, R=3, M=12, T=T, start="user", user_start=to_dev(us, "c128"), dtype="c128")
            ou = oracle.ftlm(osys(w), R=3, M=12, T=T, start="user", user_start=us)
            assert g["shape"]["vector_major"] == 1
            compare_tridiag(g, ou, 1e-10)
        finally:
            for R in (6, 3):
                for dt in ("c128", "c64"):
                    F.tune_shape(s, R, dt, -1)


def test_full_size_lanczos_sample():
    """d = 1,048,576: the first Lanczos steps of one vector against the oracle
    (complex128 to 1e-10, complex64 to 1e-5 relative in alpha and beta)."""
    w = W.lattice4x5()
    s = F.System.from_dict(w)
    M = 4
    o = oracle.ftlm(osys(w), R=1, M=M, T=T, seed=2)
    for dt, tol in (("c128", 1e-10), ("c64", 1e-5)):
        g = F.run(s, R=1, M=M, T=T, seed=2, dtype=dt)
        compare_tridiag(g, o, tol)
        try:  # the vector-major block, one pass and four
            for mp in (3, 5, 8):
                F.tune_shape(s, 1, dt, 4, 1, 1, mp)
                g = F.run(s, R=1, M=M, T=T, seed=2, dtype=dt)
                assert g["shape"]["vector_major"] == 1 and g["shape"]["passes"] == {3: 1, 5: 4, 8: 2}[mp]
                compare_tridiag(g, o, tol)
        finally:
            F.tune_shape(s, 1, dt, -1)


def test_run_rejects_bad_params():
    s = F.System.from_dict(W.square_lattice(2, 2, seed=1))
    with pytest.raises(F.FtlmError):
        F.run(s, R=0, M=5, T=T)
    with pytest.raises(F.FtlmError):
        F.run(s, R=2, M=5, T=[1.0, -1.0])
    with pytest.raises(F.FtlmError):
        F.run(s, R=2, M=5, T=T, start="basis", basis_offset=15)


@pytest.mark.parametrize("R", [1, 2, 4, 8, 16])
def test_ftlm_general_vector_major_matches_oracle(R):
    """The vector-major general plan (any spins): every vector contiguous and
    H.v over groups of V vectors -- the register cube of the top site where
    its group size divides R, else rows_vm_kernel with the largest of 8, 4, 2,
    1 (at most 4 in complex128) that divides R -- against the oracle step by
    step (complex128) and in the thermodynamics (complex64)."""
    w = random_system(np.random.default_rng(26070 + R), [2, 1, 3, 2, 1])   # d = 3*2*4*3*2 = 144
    s = F.System.from_dict(w)
    o = oracle.ftlm(osys(w), R=R, M=30, T=T, seed=8, vec_offset=1)
    g = F.run(s, R=R, M=30, T=T, seed=8, vec_offset=1, dtype="c128")
    assert g["shape"]["vector_major"] == 1 and g["shape"]["cube_bits"] == 0
    assert g["shape"]["group_vectors"] == max(v for v in (4, 2, 1) if R % v == 0)
    compare_tridiag(g, o, 1e-10)
    # the top site is s = 1/2: a register cube of its 2 rows where the group size divides R
    assert g["shape"]["site_cube"] == (2 if R % 4 == 0 else 0)
    g64 = F.run(s, R=R, M=30, T=T, seed=8, vec_offset=1, dtype="c64")
    if R % 4 == 0:  # the cube over groups of 8 vectors (complex64, 2s+1 <= 3), else of 4
        assert g64["shape"]["site_cube"] == 2 and g64["shape"]["group_vectors"] == (8 if R % 8 == 0 else 4)
    else:
        assert g64["shape"]["site_cube"] == 0 and g64["shape"]["group_vectors"] == R
    for k in KEYS:
        assert rel(g64[k], o[k], 1e-3, T >= 0.1) < 1e-4, k


@pytest.mark.parametrize("top", [2, 3, 4, 5])
def test_ftlm_site_cube_matches_oracle(top):
    """The general gather with a register cube of the top site's 2s+1 rows
    (s = 1 .. 5/2, every single-site, double-flip and pair term of the top
    site taken between cube rows or from the lower sites' neighbouring
    cubes), against the oracle step by step (complex128) and in the
    thermodynamics (complex64)."""
    w = random_system(np.random.default_rng(4100 + top), [1, 2, 1, top])   # d = 2*3*2*(top+1)
    s = F.System.from_dict(w)
    R = 8
    o = oracle.ftlm(osys(w), R=R, M=30, T=T, seed=3)
    g = F.run(s, R=R, M=30, T=T, seed=3, dtype="c128")
    assert g["shape"]["site_cube"] == top + 1 and g["shape"]["vector_major"] == 1
    compare_tridiag(g, o, 1e-10)
    g64 = F.run(s, R=R, M=30, T=T, seed=3, dtype="c64")
    assert g64["shape"]["site_cube"] == top + 1
    compare_tridiag(g64, o, 2e-5, steps=5)
    for k in KEYS:
        assert rel(g64[k], o[k], 1e-3, T >= 0.1) < 1e-4, k


def test_ftlm_site_cube_batch_matches_single_runs():
    """A batch whose systems share the top spin (s = 1, sizes 3^5 .. 3^7)
    takes the cube kernel over the prefix-summed tiles of all instances and
    gives each system's single-run result (complex128)."""
    ws = [W.chain(n, Bdir=(1.0, 0.5, 0.3)) for n in (5, 6, 7)]
    systems = [F.System.from_dict(w) for w in ws]
    R, M = 8, 20
    res = F.run_batch(systems, R=R, M=M, T=T, seed=4, dtype="c128")
    assert all(r["shape"]["site_cube"] == 3 for r in res)
    for w, r in zip(ws, res):
        o = oracle.ftlm(osys(w), R=R, M=M, T=T, seed=4)
        compare_tridiag(r, o, 1e-10)
    for s_ in systems:
        s_.close()


def test_tune_shape_vector_major_general():
    """ftlm_tune_shape with cube_bits 0 and multipass 1 forces the
    vector-major general gather: group_vectors 0 (one row a thread) or a
    cube group size, tile_cubes x 256 rows or bases per tile; invalid values
    are rejected.  Every forced shape gives the same scalars (complex128)."""
    w = random_system(np.random.default_rng(4242), [2, 1, 2, 2])   # d = 54, top site s = 1
    s = F.System.from_dict(w)
    R, M = 8, 20
    with pytest.raises(F.FtlmError):
        F.tune_shape(s, R, "c128", 0, 3, 1, 1)      # 3 does not divide 8
    with pytest.raises(F.FtlmError):
        F.tune_shape(s, R, "c128", 0, 4, 1, 2)      # multipass must be 0 or 1
    with pytest.raises(F.FtlmError):
        F.tune_shape(s, R, "c128", 0, 4, 0, 1)      # tile_cubes must be >= 1
    o = oracle.ftlm(osys(w), R=R, M=M, T=T, seed=6)
    shapes = {}
    try:
        for gv, tc in ((0, 1), (0, 4), (4, 1), (4, 2)):
            F.tune_shape(s, R, "c128", 0, gv, tc, 1)
            g = F.run(s, R=R, M=M, T=T, seed=6, dtype="c128")
            assert g["shape"]["vector_major"] == 1 and g["shape"]["site_cube"] == (3 if gv else 0)
            assert g["shape"]["tile_rows"] == 256 * tc
            compare_tridiag(g, o, 1e-10)
            shapes[(gv, tc)] = g["shape"]
        F.tune_shape(s, R, "c128", 0, 1, 2, 0)      # the row-major general kernel
        g = F.run(s, R=R, M=M, T=T, seed=6, dtype="c128")
        assert g["shape"]["vector_major"] == 0
        compare_tridiag(g, o, 1e-10)
    finally:
        F.tune_shape(s, R, "c128", -1)
        s.close()


def test_batch_of_mixed_top_spins_uses_one_row_gather():
    """A batch whose systems end in different spins has no common register
    cube: the vector-major gather with one row a thread runs it (the blocks
    fit L2), and every system's scalars match its oracle run (complex128)."""
    # d = 36, 36, 48 > M: no system exhausts its Krylov space within the M steps compared
    ws = [random_system(np.random.default_rng(700 + k), ts) for k, ts in enumerate([[1, 2, 1, 2], [2, 1, 2, 1], [3, 2, 1, 1]])]
    systems = [F.System.from_dict(w) for w in ws]
    R, M = 8, 20
    res = F.run_batch(systems, R=R, M=M, T=T, seed=2, dtype="c128")
    for w, r in zip(ws, res):
        assert r["shape"]["vector_major"] == 1 and r["shape"]["site_cube"] == 0
        compare_tridiag(r, oracle.ftlm(osys(w), R=R, M=M, T=T, seed=2), 1e-10)
    for s_ in systems:
        s_.close()
