"""The mixed-spin Mn9-like workload (Sec. III.C: a spin-5/2 centre and eight
spin-2 cube vertices, d = 2,343,750, powder average over 10 field
directions), on the general mixed-radix kernel, against the FP64 oracle."""
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


def test_full_size_sampled_rows(rng):
    """d = 2,343,750 x R = 8 (complex64): sampled rows incl. the first and last."""
    w = W.mn9(Bdir=W.dodecahedron_directions()[4])
    s = F.System.from_dict(w)
    d, R = s.dim, 8
    torch = torch_cuda()
    g = torch.Generator(device="cuda").manual_seed(3)
    x = torch.randn(d, R, dtype=torch.complex64, device="cuda", generator=g)
    y = torch.empty_like(x)
    F.apply_h(s, x, y, R, "c64")
    rows = np.unique(np.concatenate([[0, d - 1, d // 3], rng.integers(0, d, size=10)]))
    ref = sampled_rows_reference(w, x, rows)
    got = y[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert rel_l2(got, ref) < 2e-5


def test_small_mn9_ftlm_matches_oracle():
    """Centre + 3 vertices (d = 750): complex128 run to 1e-10 of the oracle,
    complex64 to 1e-4, with time-reversed pairs."""
    w = W.mn9(vertices=3, Bdir=W.dodecahedron_directions()[1])
    s = F.System.from_dict(w)
    o = oracle.ftlm(osys(w), R=6, M=40, T=T, seed=5, start="pairs")
    g = F.run(s, R=6, M=40, T=T, seed=5, start="pairs", dtype="c128")
    for k in KEYS:
        assert rel(g[k], o[k], 1e-3, T >= 0.1) < 1e-9, k
    g64 = F.run(s, R=6, M=40, T=T, seed=5, start="pairs", dtype="c64")
    for k in KEYS:
        assert rel(g64[k], o[k], 1e-3, T >= 0.1) < 1e-4, k


def test_powder_batch_matches_oracle():
    """The 10 field directions as one batch with time-reversed start pairs:
    per direction and the powder average of M_B against the oracle run
    direction by direction."""
    ws = [W.mn9(vertices=3, Bdir=u) for u in W.dodecahedron_directions()]
    systems = [F.System.from_dict(w) for w in ws]
    outs = F.run_batch(systems, R=4, M=30, T=T, seed=2, dtype="c128", start="pairs")
    refs = [oracle.ftlm(osys(w), R=4, M=30, T=T, seed=2, start="pairs") for w in ws]
    for g, o in zip(outs, refs):
        for k in KEYS:
            assert rel(g[k], o[k], 1e-3, T >= 0.1) < 1e-9, k
    avg_g = np.mean([g["M_B"] for g in outs], axis=0)
    avg_o = np.mean([o["M_B"] for o in refs], axis=0)
    assert rel(avg_g, avg_o, 1e-3, T >= 0.1) < 1e-9
