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


def test_peak_record_has_every_unit():
    """The committed probe record carries every rate the bench divides by."""
    up = bench.unit_peaks()
    for k in ("dfma_tflops", "ffma_tflops", "dmma_tflops", "tf32_tcgen05_tflops", "bf16_tcgen05_tflops"):
        assert up[k] > 0, k
    # DMMA below DFMA on this part: the FP64 forms run on DFMA
    assert up["dmma_tflops"] < up["dfma_tflops"] < up["ffma_tflops"] < up["tf32_tcgen05_tflops"]


def test_traffic_record_follows_the_kernel_source(tmp_path, monkeypatch):
    """roofline.traffic is reported only while the LU source is the one the counters
    were taken on: the committed record matches the committed source, and a changed
    source turns it into None."""
    import shutil
    v = bench.traffic_record("lu_schur", "fp64", [3, 3])
    assert v is not None and v > 0
    assert bench.traffic_record("lu_schur", "fp64", [3, 4]) is None
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    shutil.copy(bench.os.path.join(bench.ROOT, "profiles", "dram_traffic.txt"), root / "profiles")
    src = root / "paper_1605_01020_gb300" / "csrc"
    src.mkdir(parents=True)
    text = open(bench.os.path.join(bench.ROOT, "paper_1605_01020_gb300", "csrc", "iedg_assemble.cu")).read()
    (src / "iedg_assemble.cu").write_text(text)
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.traffic_record("lu_schur", "fp64", [3, 3]) == v
    (src / "iedg_assemble.cu").write_text(text + "\n// changed\n")
    assert bench.traffic_record("lu_schur", "fp64", [3, 3]) is None
