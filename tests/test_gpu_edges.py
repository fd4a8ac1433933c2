"""Edge cases of the GPU path against the FP64 oracle: one Lanczos step, the
largest vector blocks the ABI accepts, a single site (no pairs, d smaller
than any tile), zero field with and without an observable direction, and a
dimension that is not a multiple of any tile (ragged last tile)."""
import numpy as np
import pytest
from conftest import random_system
from gpu_helpers import empty_dev, osys, rel_l2, to_dev, torch_cuda

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


@pytest.mark.parametrize("w", [W.square_lattice(4, 3, seed=1), random_system(np.random.default_rng(3), [2, 1, 3])])
def test_single_lanczos_step(w):
    """M = 1: each vector contributes its Rayleigh quotient <r|H|r> alone."""
    s = F.System.from_dict(w)
    o = oracle.ftlm(osys(w), R=5, M=1, T=T, seed=4)
    g = F.run(s, R=5, M=1, T=T, seed=4, dtype="c128")
    assert list(g["M_eff"]) == [1] * 5
    assert np.allclose(g["alpha"][:, 0], o["alpha"][:, 0], rtol=1e-12)
    for k in ("lnZ", "E", "C", "M_B"):
        assert rel(g[k], o[k]) < 1e-10, k


@pytest.mark.parametrize("dtype,nvec", [("c64", 512), ("c128", 256)])
def test_largest_blocks(dtype, nvec):
    """The largest nvec the ABI accepts (512 complex64, 256 complex128)."""
    rng = np.random.default_rng(9)
    w = random_system(rng, [1, 2, 1, 3])  # d = 48
    s = F.System.from_dict(w)
    x = rng.normal(size=(s.dim, nvec)) + 1j * rng.normal(size=(s.dim, nvec))
    if dtype == "c64":
        x = x.astype(np.complex64).astype(np.complex128)
    y = empty_dev((s.dim, nvec), dtype)
    F.apply_h(s, to_dev(x, dtype), y, nvec, dtype)
    assert rel_l2(y.cpu().numpy(), oracle.apply_h(osys(w), x)) < (1e-12 if dtype == "c128" else 2e-5)
    o = oracle.ftlm(osys(w), R=nvec, M=8, T=T, seed=1)
    g = F.run(s, R=nvec, M=8, T=T, seed=1, dtype=dtype)
    for k in ("lnZ", "E", "C", "M_B"):
        assert rel(g[k], o[k], 1e-3, T >= 0.1) < (1e-10 if dtype == "c128" else 1e-4), k


@pytest.mark.parametrize("two_s", [1, 4, 5])
def test_single_site(two_s):
    """One spin (no pairs, no dipolar term): d = 2s + 1 rows, far below a tile;
    the Lanczos space is exhausted after d steps (breakdown)."""
    w = {"name": "one", "two_s": np.array([two_s], dtype=np.int32), "J": np.zeros((1, 1)),
         "d_ion": np.array([-2.0]), "e_axes": np.array([[0.3, 0.1, 0.9]]), "g": 2.0,
         "B": np.array([0.2, -0.4, 0.7]), "pos": None}
    s = F.System.from_dict(w)
    rng = np.random.default_rng(two_s)
    x = rng.normal(size=(s.dim, 3)) + 1j * rng.normal(size=(s.dim, 3))
    y = empty_dev((s.dim, 3), "c128")
    F.apply_h(s, to_dev(x, "c128"), y, 3, "c128")
    assert rel_l2(y.cpu().numpy(), oracle.apply_h(osys(w), x)) < 1e-12
    o = oracle.ftlm(osys(w), R=2, M=10, T=T, seed=2)
    g = F.run(s, R=2, M=10, T=T, seed=2, dtype="c128")
    assert list(g["M_eff"]) == list(o["M_eff"]) and max(g["M_eff"]) <= s.dim
    for k in ("lnZ", "E", "C", "M_B"):
        assert rel(g[k], o[k], 1e-3, T >= 0.1) < 1e-10, k


def test_zero_field():
    """B = 0: the observable direction defaults to z, or is given; M_B of a
    zero-field system vanishes in the exact average, and the FTLM estimate
    matches the oracle's for the same vectors."""
    w = dict(W.square_lattice(3, 3, seed=2), B=np.zeros(3))
    s = F.System.from_dict(w)
    for u in (None, np.array([1.0, 1.0, 0.0])):
        o = oracle.ftlm(osys(w), R=4, M=20, T=T, seed=3,
                        direction=None if u is None else u / np.linalg.norm(u))
        g = F.run(s, R=4, M=20, T=T, seed=3, dtype="c128", obs_dir=u)
        for k in ("lnZ", "E", "C"):
            assert rel(g[k], o[k], 1e-3, T >= 0.1) < 1e-10, k
        assert np.max(np.abs(g["M_B"] - o["M_B"])) < 1e-10 * max(1.0, np.abs(o["M_B"]).max())


def test_ragged_dimension():
    """d = 3^7 = 2187 (s = 1 chain): no power of two, so the last row tile of
    every launch shape is partial."""
    w = W.chain(7, Bdir=(0.3, -0.2, 0.9))
    s = F.System.from_dict(w)
    o = oracle.ftlm(osys(w), R=8, M=30, T=T, seed=6)
    for dt, tol in (("c128", 1e-10), ("c64", 1e-4)):
        g = F.run(s, R=8, M=30, T=T, seed=6, dtype=dt)
        for k in ("lnZ", "E", "C", "M_B"):
            assert rel(g[k], o[k], 1e-3, T >= 0.1) < tol, (dt, k)
