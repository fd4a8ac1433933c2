"""Host-side logic of bench.py (no GPU): the algorithmic flop count that
the roofline fractions divide by, pinned against a direct count over the
basis, and the per-temperature error summary."""
import itertools

import numpy as np
import pytest

import bench


def brute_force_flops(two_s, epilogue):
    """Average over every basis state of the flops its row of H costs: the
    valid flips counted one by one (a pair's s+ s- / s- s+ terms 4 flops,
    s+ s+ / s- s- 8; single-site steps by one or two levels 8; diagonal 2)."""
    q = [t + 1 for t in two_s]
    total = 0.0
    rows = list(itertools.product(*[range(k) for k in q]))
    for a in rows:
        f = 2.0 + (14.0 if epilogue else 0.0)
        for i, (ai, qi) in enumerate(zip(a, q)):
            f += 8.0 * ((ai >= 1) + (ai + 1 < qi)) + 8.0 * ((ai >= 2) + (ai + 2 < qi))
            for j in range(i + 1, len(q)):
                aj, qj = a[j], q[j]
                f += 4.0 * ((ai >= 1 and aj + 1 < qj) + (ai + 1 < qi and aj >= 1))
                f += 8.0 * ((ai >= 1 and aj >= 1) + (ai + 1 < qi and aj + 1 < qj))
        total += f
    return total / len(rows)


def test_flops_spin_half_closed_form():
    # every pair has exactly one valid flip (6 flops on average), every site one (8)
    n = 20
    assert bench.algorithmic_flops_per_sv([1] * n) == n * (n - 1) // 2 * 6 + n * 8 + 2 + 14 == 1316


@pytest.mark.parametrize("two_s", [[1, 1, 1], [2, 2, 2, 2], [1, 2, 3], [5, 4, 4], [3, 1, 4, 2]])
@pytest.mark.parametrize("epilogue", [True, False])
def test_flops_match_brute_force(two_s, epilogue):
    assert bench.algorithmic_flops_per_sv(two_s, epilogue) == pytest.approx(brute_force_flops(two_s, epilogue),
                                                                            rel=1e-12)


def test_per_t_errors_floor_and_maxima():
    T = np.array([0.05, 0.1, 1.0, 10.0])
    b = {"lnZ": np.array([1.0, 2.0, 3.0, 4.0]), "E": np.array([-1.0, -1.0, 0.0, 2.0]),
         "C": np.ones(4), "M_B": np.array([0.0, 1.0, 0.5, 0.25])}
    a = {k: v.copy() for k, v in b.items()}
    a["lnZ"][2] += 3e-6                 # relative 1e-6 at T = 1
    a["E"][2] += 2e-5                   # E = 0 there: floor 1e-3 x max|E| = 2e-3 -> 1e-2
    a["M_B"][0] += 1e-3                 # below T = 0.1: counted in max_all_T only
    e = bench.per_t_errors(a, b, T)
    assert e["lnZ"]["max_T_ge_0.1"] == pytest.approx(1e-6)
    assert e["E"]["max_T_ge_0.1"] == pytest.approx(1e-2)
    assert e["C"]["max_all_T"] == 0.0
    assert e["M_B"]["max_T_ge_0.1"] == 0.0 and e["M_B"]["max_all_T"] == pytest.approx(1.0)
    assert e["max_T_ge_0.1"] == pytest.approx(1e-2)
