"""The C-ABI library loads, exports every symbol include/ftlm.h declares, and
its host-only parts work without a GPU (argument validation happens before
any CUDA call; ftlm_sums is pure host code)."""
import os
import re

import numpy as np
import pytest

import ftlm_workloads as W
import oracle
import paper_2607_25585_gb300 as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    F.build()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ftlm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ftlm_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 10
    L = F.lib()
    for n in names:
        assert hasattr(L, n), n
    assert sorted(F.EXPORTS) == names


def test_version():
    assert "sm_103a" in F.version()


def test_struct_layouts_match_header(tmp_path):
    """The ctypes structures of the binding have the field offsets and sizes
    that a C compiler gives the structs of include/ftlm.h (a plain C program
    built with gcc prints them)."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"ftlm_run_params": F.RunParams, "ftlm_result": F.Result, "ftlm_constants": F.Constants}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ftlm.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = 0
    for ln in out:
        if not ln.strip():
            continue
        cname, field, val = ln.split()
        py = structs[cname]
        expect = ctypes.sizeof(py) if field == "sizeof" else getattr(py, field).offset
        assert int(val) == expect, (cname, field)
        seen += 1
    assert seen == sum(len(p._fields_) + 1 for p in structs.values())


def test_run_params_reorth_validated_on_host():
    """ftlm_run_params.reorth takes 0 (the three-term recurrence) or 1 (full
    re-orthogonalisation); anything else is rejected before the library
    looks at the system or touches the GPU."""
    import ctypes
    keep = []
    T = W.temperatures()
    p = F._params(2, 5, T, 0, 0, "c64", "random", 0, None, None, 0.0, False, False, None, keep)
    r, _ = F._result(2, 5, len(T), keep)
    for bad in (2, -1):
        p.reorth = bad
        assert F.lib().ftlm_run(None, ctypes.byref(p), ctypes.byref(r)) == 1
        assert "reorth" in F.lib().ftlm_last_error().decode()
    p.reorth = 1
    assert F.lib().ftlm_run(None, ctypes.byref(p), ctypes.byref(r)) == 1
    assert "system is NULL" in F.lib().ftlm_last_error().decode()


def test_binding_checks_blocks_before_the_library():
    """The Python binding refuses a tensor block that is not on a CUDA device,
    not contiguous, of the wrong element size for the dtype, or too small for
    [dim][nvec], before any pointer reaches the library (no GPU needed: the
    checks run on CPU tensors)."""
    torch = pytest.importorskip("torch")
    ok = torch.zeros(8, 4, dtype=torch.complex64)
    with pytest.raises(F.FtlmError, match="device block"):
        F._check_block(ok, 8, 4, "c64")

    class Fake:  # a device tensor stand-in: only the attributes the check reads
        def __init__(self, t, dev="cuda"):
            self.t, self.device = t, torch.device(dev)

        def is_contiguous(self):
            return self.t.is_contiguous()

        def element_size(self):
            return self.t.element_size()

        def numel(self):
            return self.t.numel()

    F._check_block(Fake(ok), 8, 4, "c64")
    F._check_block(12345, 8, 4, "c64")                  # raw pointers pass through
    with pytest.raises(F.FtlmError, match="do not match"):
        F._check_block(Fake(ok), 8, 4, "c128")           # complex64 storage passed as complex128
    with pytest.raises(F.FtlmError, match="elements"):
        F._check_block(Fake(ok), 8, 5, "c64")            # too small for [8][5]
    with pytest.raises(F.FtlmError, match="contiguous"):
        F._check_block(Fake(torch.zeros(4, 8, dtype=torch.complex64).t()), 8, 4, "c64")


@pytest.mark.parametrize("kw,msg", [
    (dict(two_s=[1, 0]), "two_s"),
    (dict(two_s=[1, 16]), "two_s"),
    (dict(two_s=[1, 1], pos=np.zeros((2, 3))), "coincide"),
    (dict(two_s=[2, 2], d_ion=[1.0, 0.0], e_axes=np.zeros((2, 3))), "e_axes"),
    (dict(two_s=[1, 1], B=[0.0, np.nan, 0.0]), "finite"),
    (dict(two_s=[1] * 37), "2^36"),
])
def test_invalid_systems_rejected_on_host(kw, msg):
    with pytest.raises(F.FtlmError) as e:
        F.System(**kw)
    assert msg in str(e.value)


def test_sums_match_oracle(rng):
    """ftlm_sums (implicit QL on the host) against the oracle's sums (cyclic
    Jacobi) on the same tridiagonal data."""
    s = oracle.System(**{k: v for k, v in W.ring(N=4, two_s=2).items() if k != "name"})
    T = W.temperatures()
    o = oracle.ftlm(s, R=4, M=30, T=T, seed=3)
    r = F.sums(o["alpha"], o["beta"], o["p"], o["M_eff"], s.dim, s.g, T)
    for k in ("lnZ", "E", "C", "M_B", "M_B_imag"):
        ref = o[k]
        scale = np.maximum(np.abs(ref), 1e-6 * np.abs(ref).max() + 1e-300)
        assert np.max(np.abs(r[k] - ref) / scale) < 1e-10, k
    assert abs(r["E0"] - o["E0"]) < 1e-12 * abs(o["E0"])


def test_sums_reject_bad_input():
    with pytest.raises(F.FtlmError):
        F.sums(np.zeros((1, 3)), np.zeros((1, 3)), np.zeros((1, 3)), [4], 8, 2.0, [1.0])
    with pytest.raises(F.FtlmError):
        F.sums(np.zeros((1, 3)), np.zeros((1, 3)), np.zeros((1, 3)), [2], 8, 2.0, [0.0])


def test_sums_many_runs_deterministic_and_per_run(rng):
    """The runs' eigenproblems and the temperatures are spread over host
    threads: the result must not depend on that (bitwise equal on repeat and
    equal to the runs merged one at a time in the same order), and an error
    names the run it comes from."""
    R, M = 40, 60
    # weak disorder (extended Ritz vectors), so that every temperature's
    # weights are well conditioned
    a = 0.1 * rng.normal(size=(R, M))
    b = 1.0 + 0.1 * np.abs(rng.normal(size=(R, M)))
    p = rng.normal(size=(R, M)) + 1j * rng.normal(size=(R, M))
    me = rng.integers(1, M + 1, size=R).astype(np.int32)
    T = np.geomspace(0.05, 50.0, 33)
    r1 = F.sums(a, b, p, me, 4096, 2.0, T)
    r2 = F.sums(a, b, p, me, 4096, 2.0, T)
    for k in ("lnZ", "E", "C", "M_B", "M_B_imag"):
        assert np.array_equal(r1[k], r2[k]), k
    # Eqs. 4-5 from the per-run Ritz data, merged by hand
    ev = [np.linalg.eigh(np.diag(a[r, :me[r]]) + np.diag(b[r, :me[r] - 1], 1) + np.diag(b[r, :me[r] - 1], -1))
          for r in range(R)]
    E0 = min(w.min() for w, _ in ev)
    for t, Tt in enumerate(T):
        z = e1 = orr = 0.0
        for r, (w, U) in enumerate(ev):
            bz = np.exp(-(w - E0) / Tt)
            z += np.sum(U[0] ** 2 * bz)
            e1 += np.sum(U[0] ** 2 * bz * w)
            orr += np.sum(bz * U[0] * (np.conj(p[r, :me[r]]) @ U).real)
        assert abs(r1["E"][t] - e1 / z) < 1e-9 * max(1.0, abs(e1 / z)), t
        assert abs(r1["M_B"][t] + 2.0 * orr / z) < 1e-9 * max(1.0, abs(orr / z)), t
    bad = a.copy()
    bad[27, 0] = np.nan
    with pytest.raises(F.FtlmError, match="run 27"):
        F.sums(bad, b, p, me, 4096, 2.0, T)


def test_sums_sym_match_oracle(rng):
    """ftlm_sums_sym (host-only) reproduces the oracle's symmetric estimator
    from the same per-vector data."""
    from conftest import random_system, oracle_system
    w = random_system(rng, [1, 2, 1, 1])
    T = np.array([0.1, 0.5, 2.0, 10.0])
    o = oracle.sftlm(oracle_system(w), R=3, M=12, T=T, seed=3)
    mb, mbi = F.sums_sym(o["alpha"], o["beta"], o["O"], o["M_eff"], w["g"], T)
    assert np.allclose(mb, o["M_B_sym"], rtol=1e-11, atol=1e-13)
    assert np.allclose(mbi, o["M_B_sym_imag"], rtol=1e-9, atol=1e-12)


def test_sums_sym_many_runs_match_definition(rng):
    """ftlm_sums_sym with the runs and temperatures spread over host threads:
    bitwise equal on repeat, and equal to Eqs. E-2-G/H written out with numpy
    (y = U e^{-beta eps/2} U_0, num = y^T O y, den = sum e^{-beta eps} U_0^2)."""
    R, M = 24, 16
    a = 0.1 * rng.normal(size=(R, M))
    b = 1.0 + 0.1 * np.abs(rng.normal(size=(R, M)))
    O = rng.normal(size=(R, M, M)) + 1j * rng.normal(size=(R, M, M))
    O = 0.5 * (O + np.conj(np.transpose(O, (0, 2, 1))))  # Hermitian, as <v_i|O|v_j> is
    me = rng.integers(2, M + 1, size=R).astype(np.int32)
    T = np.geomspace(0.1, 20.0, 17)
    g = 2.0
    mb1, mbi1 = F.sums_sym(a, b, O, me, g, T)
    mb2, mbi2 = F.sums_sym(a, b, O, me, g, T)
    assert np.array_equal(mb1, mb2) and np.array_equal(mbi1, mbi2)
    ev = [np.linalg.eigh(np.diag(a[r, :me[r]]) + np.diag(b[r, :me[r] - 1], 1) + np.diag(b[r, :me[r] - 1], -1))
          for r in range(R)]
    E0 = min(w.min() for w, _ in ev)
    for t, Tt in enumerate(T):
        num, den = 0.0, 0.0
        for r, (w, U) in enumerate(ev):
            m = me[r]
            h = np.exp(-0.5 * (w - E0) / Tt)
            y = U @ (h * U[0])
            num += y @ O[r, :m, :m] @ y
            den += np.sum(h * h * U[0] ** 2)
        ref = -g * num / den
        assert abs(mb1[t] - ref.real) < 1e-10 * max(1.0, abs(ref)), t
        assert abs(mbi1[t] - ref.imag) < 1e-10 * max(1.0, abs(ref)), t


@pytest.mark.parametrize("lam", [1e-170, 1e-3, 1e3, 1e170])
def test_sums_scale_invariance(rng, lam):
    """Scaling alpha, beta and T by the same factor scales E by it and leaves
    ln Z and M_B unchanged (Eqs. 4-5 depend on (eps - E0) / T only).  At
    1e+-170 the squares in the eigensolver's rotations would overflow or
    underflow, so this also checks that they are formed without squaring
    there."""
    R, M = 6, 40
    a = 0.1 * rng.normal(size=(R, M))
    b = 1.0 + 0.1 * np.abs(rng.normal(size=(R, M)))
    p = rng.normal(size=(R, M)) + 1j * rng.normal(size=(R, M))
    me = np.full(R, M, dtype=np.int32)
    T = np.geomspace(0.1, 10.0, 7)
    r1 = F.sums(a, b, p, me, 4096, 2.0, T)
    r2 = F.sums(lam * a, lam * b, p, me, 4096, 2.0, lam * T)
    assert np.allclose(r2["E"] / lam, r1["E"], rtol=1e-11, atol=1e-13)
    assert np.allclose(r2["lnZ"], r1["lnZ"], rtol=1e-11, atol=1e-11)
    assert np.allclose(r2["M_B"], r1["M_B"], rtol=1e-10, atol=1e-12)
