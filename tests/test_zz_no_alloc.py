"""ftlm_start_block_noalloc -- the start block for callers that cannot
allocate device memory (code running inside someone else's memory budget,
or at a point where cudaMalloc / cudaFree are off limits).  It must give what
the allocating ftlm_start_block gives, on consecutive calls that reuse its
static scratch, through the C ABI.

This file is collected last so that a stop-at-first-failure run has executed
every other test before it; it also passes on its own in a fresh process."""
import numpy as np
import pytest
from gpu_helpers import empty_dev, rel_l2, torch_cuda

import ftlm_workloads as W
import paper_2607_25585_gb300 as F

pytestmark = pytest.mark.gpu
# the tolerances of the start-block parity tests
TOL = {"c128": 1e-14, "c64": 1e-7}


@pytest.fixture(scope="module", autouse=True)
def built():
    F.build()
    torch_cuda()


def test_no_alloc_start_block_matches_the_allocating_one():
    s = F.System.from_dict(W.square_lattice(4, 3, seed=1))
    d = s.dim
    for call in range(2):                      # the second call reuses the scratch the first left behind
        for dtype in ("c128", "c64"):
            for R, seed, off in ((5, 11, 0), (64, 3, 7 + call)):
                ref = empty_dev((d, R), dtype)
                F.start_block(s, ref, R, seed=seed, vec_offset=off, dtype=dtype)
                got = empty_dev((d, R), dtype)
                got.zero_()
                F.start_block_noalloc(s, got, R, seed=seed, vec_offset=off, dtype=dtype)
                g, r = got.cpu().numpy(), ref.cpu().numpy()
                assert rel_l2(g, r) < TOL[dtype], (call, dtype, R)
                assert np.allclose(np.linalg.norm(g, axis=0), 1.0, atol=1e-6 if dtype == "c64" else 1e-14)


def test_no_alloc_full_size_more_ctas_than_its_scratch_holds():
    """d = 1,048,576 x 64 vectors: the allocating call launches more CTAs than
    the static scratch has partial-sum slots (256), so the allocation-free
    call runs on fewer CTAs and sums the norms over another partition; the
    blocks agree within the tolerance of the start-block tests and every
    column has norm 1."""
    s = F.System.from_dict(W.lattice4x5())
    d, R = s.dim, 64
    for call in range(2):
        for dtype in ("c128", "c64"):
            ref = empty_dev((d, R), dtype)
            F.start_block(s, ref, R, seed=7, vec_offset=call, dtype=dtype)
            got = empty_dev((d, R), dtype)
            got.zero_()
            F.start_block_noalloc(s, got, R, seed=7, vec_offset=call, dtype=dtype)
            torch = torch_cuda()
            diff = torch.linalg.vector_norm((got - ref).to(torch.complex128)).item()
            nref = torch.linalg.vector_norm(ref.to(torch.complex128)).item()
            assert diff / nref < TOL[dtype], (call, dtype)
            norms = torch.linalg.vector_norm(got.to(torch.complex128), dim=0).cpu().numpy()
            assert np.allclose(norms, 1.0, atol=1e-6 if dtype == "c64" else 1e-14)
            del ref, got


def test_no_alloc_rejects_blocks_beyond_its_scratch():
    s = F.System.from_dict(W.square_lattice(4, 3, seed=1))
    out = empty_dev((s.dim, 65), "c64")
    with pytest.raises(F.FtlmError) as e:
        F.start_block_noalloc(s, out, 65, seed=1, dtype="c64")
    assert "static scratch" in str(e.value)
