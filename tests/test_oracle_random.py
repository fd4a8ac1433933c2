"""Pins for the oracle's random start vectors (Eq. 2: complex Gaussian
components with zero mean), drawn with Philox4x32-10 + Box-Muller."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t, 16) for t in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat())
def test_philox_known_answers(ctr, key, expect):
    out = oracle.philox4x32_10(ctr, key)
    assert [int(x) for x in out] == expect


def test_start_vectors_normalised_and_reproducible():
    a = oracle.start_vectors(1000, 3, seed=7)
    b = oracle.start_vectors(1000, 3, seed=7)
    assert np.array_equal(a, b)
    assert np.allclose(np.linalg.norm(a, axis=0), 1.0, atol=1e-14)
    # column k with offset o is vector number o + k: a shifted window reproduces columns
    c = oracle.start_vectors(1000, 2, seed=7, vec_offset=1)
    assert np.array_equal(c, a[:, 1:])
    # another seed gives another vector
    assert np.abs(oracle.start_vectors(1000, 1, seed=8)[:, 0] - a[:, 0]).max() > 0.01


def test_start_vectors_are_gaussian():
    """Components of sqrt(d) r: re and im ~ N(0, 1/2) (unit vector), mean 0,
    Gaussian kurtosis 3, re/im uncorrelated, vectors nearly orthogonal."""
    d = 200_000
    r = oracle.start_vectors(d, 2, seed=0)
    z = r[:, 0] * np.sqrt(d)
    for comp in (z.real, z.imag):
        assert abs(comp.mean()) < 5 * np.sqrt(0.5 / d)
        assert abs(comp.var() - 0.5) < 0.01
        k = ((comp - comp.mean()) ** 4).mean() / comp.var() ** 2
        assert abs(k - 3.0) < 0.1   # a uniform marginal would give 1.8
    assert abs(np.corrcoef(z.real, z.imag)[0, 1]) < 0.02
    # a radius mistake in Box-Muller shows up in the radial law: |z|^2 ~ Exp(1)
    e = np.abs(z) ** 2
    for q in (0.1, 0.5, 0.9):
        assert abs(np.quantile(e, q) - (-np.log(1 - q))) < 0.02
    assert abs(np.vdot(r[:, 0], r[:, 1])) < 5 / np.sqrt(d)
