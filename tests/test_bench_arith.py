"""The benchmark's algorithmic work per apply (the numerators of its roofline fractions):
canonical FLOPs = 2 (p+1)^4 per 1D pass per scalar field per element (54 passes on the fly,
36 cached) plus 230 / 150 FLOP per Gauss point, and compulsory bytes = u, du, v (on the fly)
or du, v and the 10-value point cache (cached), checked against values computed by hand for
the benchmark workloads."""
import pytest

import bench
import nhmf_inputs as inp


@pytest.mark.parametrize("name, otf_gflop, cached_gflop, cached_mb", [
    ("q2_64_clamp", 3.92, 2.59, 669.3),      # 262,144 Q2 elements, 7,077,888 points, 6,440,067 DoFs
    ("q4_32_clamp", 3.15, 2.09, 430.5),      # 32,768 Q4 elements, 4,096,000 points
    ("q3_48_compress", 4.69, 3.10, 712.6),   # 110,592 Q3 elements, 7,077,888 points
    ("q4_64_compress", 25.2, 16.7, 3436.5),  # 262,144 Q4 elements, 32,768,000 points
])
def test_canonical_flops_and_bytes(name, otf_gflop, cached_gflop, cached_mb):
    w = inp.WORKLOADS[name]
    n = w.degree + 1
    E, qp = w.n_elements, w.n_qp
    assert E == w.n_el ** 3 and qp == E * n ** 3
    assert bench.canonical_flops(w, "otf") == E * 54 * 2 * n ** 4 + qp * 230
    assert bench.canonical_flops(w, "cached") == E * 36 * 2 * n ** 4 + qp * 150
    assert bench.canonical_flops(w, "otf") / 1e9 == pytest.approx(otf_gflop, rel=6e-3)
    assert bench.canonical_flops(w, "cached") / 1e9 == pytest.approx(cached_gflop, rel=6e-3)
    assert bench.compulsory_bytes(w, "otf", 8) == 3 * 8 * w.n_dofs
    assert bench.compulsory_bytes(w, "cached", 8) == 2 * 8 * w.n_dofs + 10 * 8 * qp
    assert bench.compulsory_bytes(w, "cached", 8) / 1e6 == pytest.approx(cached_mb, rel=1e-3)


def test_fp64_peak_is_the_unit_count_at_the_maximum_clock():
    # 152 SMs x 2 FP64 FMA per clock x 2 FLOP x 2070 MHz
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(152 * 2 * 2 * 2070e6 / 1e12)
