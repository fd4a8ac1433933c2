"""GPU parity of the time-reversal operator and of FTLM with pairs of
mutually time-reversed random vectors (Sec. II.B; tau = 1 in Sec. III)
against the FP64 oracle, through the C ABI.  Tolerances as in the matvec and
FTLM tests: the operator and the start blocks are exact up to rounding and
the libm/CUDA ulp differences of log and sincospi (1e-14 complex128, 1e-7
complex64); tridiagonal data 1e-10 over the first 20 steps (complex128)."""
import numpy as np
import pytest
from conftest import random_system
from gpu_helpers import empty_dev, osys, rel_l2, to_dev, torch_cuda

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


def systems(rng):
    return {"mixed": random_system(rng, [1, 2, 3, 5, 1]),        # general digits, d = 576
            "lattice4x3": W.square_lattice(4, 3, seed=1)}        # s = 1/2: the popcount path


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("name", ["mixed", "lattice4x3"])
def test_time_reverse_matches_oracle(name, dtype, rng):
    w = systems(rng)[name]
    s = F.System.from_dict(w)
    x = rng.normal(size=(s.dim, 3)) + 1j * rng.normal(size=(s.dim, 3))
    if dtype == "c64":
        x = x.astype(np.complex64).astype(np.complex128)
    y = empty_dev((s.dim, 3), dtype)
    F.time_reverse(s, to_dev(x, dtype), y, 3, dtype)
    assert rel_l2(y.cpu().numpy(), oracle.time_reverse(osys(w), x)) < (1e-15 if dtype == "c128" else 1e-7)


def test_time_reverse_rejects_overlap():
    s = F.System.from_dict(W.square_lattice(2, 2, seed=1))
    torch = torch_cuda()
    x = torch.zeros(s.dim, 2, dtype=torch.complex64, device="cuda")
    with pytest.raises(F.FtlmError):
        F.time_reverse(s, x, x, 2, "c64")


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("name", ["mixed", "lattice4x3"])
def test_start_pairs_matches_oracle(name, dtype, rng):
    w = systems(rng)[name]
    s = F.System.from_dict(w)
    for R, off in ((6, 0), (5, 3)):  # an odd offset starts with a reversed vector
        out = empty_dev((s.dim, R), dtype)
        F.start_pairs(s, out, R, seed=11, vec_offset=off, dtype=dtype)
        ref = oracle.start_pairs(osys(w), R, seed=11, vec_offset=off)
        assert rel_l2(out.cpu().numpy(), ref) < (1e-14 if dtype == "c128" else 1e-7)


def compare_tridiag(g, o, tol, steps=20):
    assert list(g["M_eff"]) == list(o["M_eff"])
    for r in range(o["alpha"].shape[0]):
        m = min(o["M_eff"][r], steps)
        sa = np.abs(o["alpha"][r, :m]).max()
        assert np.max(np.abs(g["alpha"][r, :m] - o["alpha"][r, :m])) < tol * sa
        assert np.max(np.abs(g["beta"][r, : m - 1] - o["beta"][r, : m - 1])) < tol * sa
        assert np.max(np.abs(g["p"][r, :m] - o["p"][r, :m])) < tol * max(1.0, np.abs(o["p"][r, :m]).max())


@pytest.mark.parametrize("name", ["mixed", "lattice4x3"])
def test_ftlm_pairs_matches_oracle(name, rng):
    """The whole run with time-reversed pairs (vector-major gather for the
    lattice, general kernel for the mixed system) against the oracle."""
    w = systems(rng)[name]
    s = F.System.from_dict(w)
    o = oracle.ftlm(osys(w), R=6, M=30, T=T, seed=5, vec_offset=2, start="pairs")
    g = F.run(s, R=6, M=30, T=T, seed=5, vec_offset=2, start="pairs", dtype="c128")
    compare_tridiag(g, o, 1e-10)
    for k in KEYS:
        assert rel(g[k], o[k], 1e-3, T >= 0.1) < 1e-9, k
    g64 = F.run(s, R=6, M=30, T=T, seed=5, vec_offset=2, start="pairs", dtype="c64")
    for k in KEYS:
        assert rel(g64[k], o[k], 1e-3, T >= 0.1) < 1e-4, k


def test_reversed_partner_sees_reversed_field(rng):
    """On the GPU: the odd vectors of a pairs run at field B have the alpha,
    beta of the plain random vectors at field -B (Theta H(B) Theta^-1 = H(-B))."""
    w = W.square_lattice(4, 3, seed=1)
    wm = dict(w, B=-np.asarray(w["B"]))
    g = F.run(F.System.from_dict(w), R=4, M=15, T=T, seed=7, start="pairs", dtype="c128")
    h = F.run(F.System.from_dict(wm), R=2, M=15, T=T, seed=7, start="random", dtype="c128")
    sa = np.abs(h["alpha"]).max()
    assert np.max(np.abs(g["alpha"][1::2] - h["alpha"])) < 1e-10 * sa
    assert np.max(np.abs(g["beta"][1::2, :14] - h["beta"][:, :14])) < 1e-10 * sa
