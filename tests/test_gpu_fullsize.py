"""The benchmark workloads at their full sizes on the GPU path.

* The open 4x4 lattice (d = 65,536, R = 50, M = 150, complex128): the whole
  FTLM run against the FP64 oracle with the same Philox vectors.
* The open 4x5 lattice (d = 1,048,576, R = 64, M = 200): the batched FP32
  path (complex64 vectors, FP32 matvec, FP64 scalars) against the same run in
  complex128 (the FP64 GPU path, itself checked against the oracle at every
  smaller size and at full size on sampled rows and the first steps):
  ln Z, E, C, M_B within 1e-4 relative for T >= 0.1 K.
* The 2 x 13 ladder (d = 67,108,864): the vector-major gather the runs use,
  through ftlm_apply_h with one vector (whose row-major and vector-major
  layouts coincide), on sampled rows against the oracle's columns; and the
  first Lanczos scalars of a vector-major run against the same quantities
  formed from the oracle's start vector.

Relative errors of quantities that pass through zero take a floor of 1e-3
of their maximum over T."""
import numpy as np
import pytest
from gpu_helpers import osys, rel_l2, sampled_rows_reference, torch_cuda

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


@pytest.mark.slow
def test_lattice4x4_full_run_matches_oracle():
    spec = W.WORKLOADS["lattice4x4"]
    w = spec["system"]()
    s = F.System.from_dict(w)
    R, M = spec["R"], spec["M"]
    g = F.run(s, R=R, M=M, T=T, seed=spec["seed"], dtype="c128")
    o = oracle.ftlm(osys(w), R=R, M=M, T=T, seed=spec["seed"])
    assert list(g["M_eff"]) == list(o["M_eff"])
    for r in range(R):  # the steps before the first Ritz value converges
        sa = np.abs(o["alpha"][r, :20]).max()
        assert np.max(np.abs(g["alpha"][r, :20] - o["alpha"][r, :20])) < 1e-10 * sa
        assert np.max(np.abs(g["beta"][r, :19] - o["beta"][r, :19])) < 1e-10 * sa
    for k in KEYS:
        assert rel(g[k], o[k], 1e-3, T >= 0.1) < 1e-10, k
    assert abs(g["E0"] - o["E0"]) < 1e-10 * abs(o["E0"])


def c64_vs_c128(spec, M=None):
    w = spec["system"]()
    s = F.System.from_dict(w)
    R, M = spec["R"], M or spec["M"]
    g64 = F.run(s, R=R, M=M, T=T, seed=spec["seed"], dtype="c64")
    g128 = F.run(s, R=R, M=M, T=T, seed=spec["seed"], dtype="c128")
    s.close()
    return g64, g128


@pytest.mark.slow
def test_lattice4x5_fp32_within_1e4_of_fp64():
    g64, g128 = c64_vs_c128(W.WORKLOADS["lattice4x5"])
    assert g64["shape"]["vector_major"] == 1 and g128["shape"]["vector_major"] == 1
    cold = T >= 0.1
    for k in KEYS:
        assert rel(g64[k], g128[k], 1e-3, cold) < 1e-4, k


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_ladder_vector_major_sampled_rows(dtype, rng):
    w = W.ladder2x13()
    s = F.System.from_dict(w)
    d = s.dim
    torch = torch_cuda()
    tdt = torch.complex64 if dtype == "c64" else torch.complex128
    g = torch.Generator(device="cuda").manual_seed(11)
    x = torch.randn(d, 1, dtype=tdt, device="cuda", generator=g)
    y = torch.empty_like(x)
    F.apply_h(s, x, y, 1, dtype)
    rows = np.unique(np.concatenate([[0, 1, 31, 32, d // 2, d - 2, d - 1], rng.integers(0, d, size=12)]))
    ref = sampled_rows_reference(w, x, rows)
    got = y[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert rel_l2(got, ref) < (2e-5 if dtype == "c64" else 1e-12)


def test_ladder_vector_major_run_first_steps():
    """A two-step run (R = 1) on the 2 x 13 ladder takes the vector-major
    gather; its alpha_0, beta_0 and p_0 equal <v0|H v0>, |H v0 - alpha_0 v0|
    and <v0|u.S v0> with v0 the oracle's start vector (Philox + Box-Muller,
    normalised in FP64) and H v0, u.S v0 formed by ftlm_apply_h and
    ftlm_apply_sdir in complex128 (checked above on sampled rows)."""
    w = W.ladder2x13()
    s = F.System.from_dict(w)
    d = s.dim
    torch = torch_cuda()
    v0 = oracle.start_vectors(d, 1, seed=5)
    g = F.run(s, R=1, M=2, T=T, seed=5, dtype="c128")
    assert g["shape"]["vector_major"] == 1
    x = torch.from_numpy(np.ascontiguousarray(v0)).cuda()
    hx = torch.empty_like(x)
    F.apply_h(s, x, hx, 1, "c128")
    ux = torch.empty_like(x)
    F.apply_sdir(s, x, ux, 1, "c128")
    a0 = torch.vdot(x[:, 0], hx[:, 0]).real.item()
    b0 = torch.linalg.vector_norm(hx[:, 0] - a0 * x[:, 0]).item()
    p0 = torch.vdot(x[:, 0], ux[:, 0]).item()
    # errors on the scale of H (alpha_0 of a random vector is tr H / d plus
    # noise of order beta_0 / sqrt(d), here ~1e-4 of beta_0)
    scale = max(abs(a0), b0)
    assert abs(g["alpha"][0, 0] - a0) < 1e-10 * scale
    assert abs(g["beta"][0, 0] - b0) < 1e-10 * scale
    assert abs(g["p"][0, 0] - p0) < 1e-10 * max(1.0, abs(p0))
    g64 = F.run(s, R=1, M=2, T=T, seed=5, dtype="c64")
    assert g64["shape"]["vector_major"] == 1
    assert abs(g64["alpha"][0, 0] - a0) < 1e-5 * scale
    assert abs(g64["beta"][0, 0] - b0) < 1e-5 * scale


def test_general_block_beyond_l2_first_steps_and_autotune():
    """An s = 1 chain of 12 sites (d = 531,441) with R = 30 complex128
    vectors: its block (255 MB) exceeds L2 and no register-cube group size
    (4) divides R, so a run takes the row-major general gather by default;
    alpha_0, beta_0, p_0 of every vector equal the
    quantities formed from the oracle's start vectors with ftlm_apply_h and
    ftlm_apply_sdir.  The autotuner (which also times the vector-major
    general gather) then picks a shape whose run gives the same scalars."""
    w = max(W.WORKLOADS["chains_s1_x24"]["system"](), key=lambda v: int(np.prod(v["two_s"] + 1)))
    s = F.System.from_dict(w)
    d, R = s.dim, 30
    assert d == 3 ** 12
    torch = torch_cuda()
    g = F.run(s, R=R, M=2, T=T, seed=7, dtype="c128")
    assert g["shape"]["vector_major"] == 0 and g["shape"]["cube_bits"] == 0
    x = torch.from_numpy(np.ascontiguousarray(oracle.start_vectors(d, R, seed=7))).cuda()
    hx = torch.empty_like(x)
    F.apply_h(s, x, hx, R, "c128")
    ux = torch.empty_like(x)
    F.apply_sdir(s, x, ux, R, "c128")
    a0 = torch.sum(x.conj() * hx, dim=0).real
    b0 = torch.linalg.vector_norm(hx - a0[None, :] * x, dim=0)
    p0 = torch.sum(x.conj() * ux, dim=0)
    a0, b0, p0 = a0.cpu().numpy(), b0.cpu().numpy(), p0.cpu().numpy()
    scale = np.maximum(np.abs(a0), b0)
    assert np.all(np.abs(g["alpha"][:, 0] - a0) < 1e-10 * scale)
    assert np.all(np.abs(g["beta"][:, 0] - b0) < 1e-10 * scale)
    assert np.all(np.abs(g["p"][:, 0] - p0) < 1e-10 * np.maximum(1.0, np.abs(p0)))
    try:
        t = F.run(s, R=R, M=2, T=T, seed=7, dtype="c128", autotune=True)
        assert t["shape"]["cube_bits"] == 0
        for k in ("alpha", "beta"):
            assert np.max(np.abs(t[k] - g[k])) < 1e-10 * scale.max(), k
    finally:
        F.tune_shape(s, R, "c128", -1)
        s.close()


def test_site_cube_chain_first_steps():
    """An s = 1 chain of 11 sites (d = 177,147, a block of 8 complex128
    vectors fits L2): the run takes the general gather with a register cube
    of the top site's 3 rows; alpha_0, beta_0, p_0 of every vector equal the
    quantities formed from the oracle's start vectors with ftlm_apply_h and
    ftlm_apply_sdir (complex128), and within FP32 rounding in complex64."""
    w = W.chain(11, Bdir=(1.0, 0.5, 0.3))
    s = F.System.from_dict(w)
    d, R = s.dim, 8
    torch = torch_cuda()
    x = torch.from_numpy(np.ascontiguousarray(oracle.start_vectors(d, R, seed=9))).cuda()
    hx = torch.empty_like(x)
    F.apply_h(s, x, hx, R, "c128")
    ux = torch.empty_like(x)
    F.apply_sdir(s, x, ux, R, "c128")
    a0 = torch.sum(x.conj() * hx, dim=0).real
    b0 = torch.linalg.vector_norm(hx - a0[None, :] * x, dim=0)
    p0 = torch.sum(x.conj() * ux, dim=0)
    a0, b0, p0 = a0.cpu().numpy(), b0.cpu().numpy(), p0.cpu().numpy()
    scale = np.maximum(np.abs(a0), b0)
    for dtype, tol in (("c128", 1e-10), ("c64", 1e-5)):
        g = F.run(s, R=R, M=2, T=T, seed=9, dtype=dtype)
        assert g["shape"]["site_cube"] == 3, dtype
        assert np.all(np.abs(g["alpha"][:, 0] - a0) < tol * scale), dtype
        assert np.all(np.abs(g["beta"][:, 0] - b0) < tol * scale), dtype
        assert np.all(np.abs(g["p"][:, 0] - p0) < tol * np.maximum(1.0, np.abs(p0))), dtype
    s.close()
