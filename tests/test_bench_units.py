"""The bench line's unit counts: flops and algorithmic bytes of one prism apply, checked against
counts taken from the sum-factorised contraction's structure and against the numbers quoted for
the 64x64x4 benchmark mesh at P = 6 (32,768 prisms, 3,705,625 nodes)."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 6])
def test_apply_flops_follow_the_contraction(bench, P):
    NT, NZ = (P + 1) * (P + 2) // 2, P + 1
    QT, QZ = (P + 1) ** 2, P + 1
    vertical = 2 * NT * QZ * NZ              # U and W from the nodal values
    triangle = 3 * QT * NT * QZ              # ur, us from U; ut from W
    factors = 9 * QT * QZ                    # the symmetric 3x3 factors per point
    # transposed stages mirror the forward ones
    assert bench.apply_flops_per_elem(P) == 2 * (2 * vertical + 2 * triangle + factors)


def test_benchmark_mesh_counts(bench):
    E, N = 32768, 3705625
    assert bench.apply_flops_per_elem(6) == 132398
    assert bench.apply_flops_per_elem(6) * E == 4338417664
    # FP64: x and y, FP64 factors, int32 map
    assert bench.apply_bytes(6, E, N) == 2 * N * 8 + E * 6 * 343 * 8 + E * 196 * 4 == 624472464
    # tensor-core form: FP32 x and y, BF16 factors
    assert bench.apply_bytes(6, E, N, word=4, gword=2) == 2 * N * 4 + E * 6 * 343 * 2 + E * 196 * 4
    assert bench.levels_for(6) == [6, 3, 1] and bench.levels_for(2) == [2, 1]
