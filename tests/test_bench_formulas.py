"""The algorithmic flop counts the benchmark divides by (fixed dense-count formulas
for assembly + q-elimination and for the partial LU / Schur complement) against the
per-element totals tabulated for p = 2, 3, 4 in 3D."""
import pytest

import bench


@pytest.mark.parametrize("p,a4a5,a6,total", [(2, 4.33e7, 1.10e7, 5.44e7), (3, 4.64e8, 1.30e8, 5.95e8),
                                               (4, 3.03e9, 8.47e8, 3.87e9)])
def test_flop_formulas(p, a4a5, a6, total):
    m, Np = 5, (p + 1) ** 3
    Nb = Np - (p - 1) ** 3
    f45 = bench.a4a5_flops(3, p, p + 2)
    f6 = bench.a6_flops(m * Np, m * Nb)
    assert abs(f45 / a4a5 - 1) < 0.01
    assert abs(f6 / a6 - 1) < 0.01
    assert abs((f45 + f6) / total - 1) < 0.01


def test_assembly_actual_count_below_dense_count():
    for p in (2, 3, 4):
        assert bench.assemble_actual_flops(3, p, p + 2) < bench.a4a5_flops(3, p, p + 2)
