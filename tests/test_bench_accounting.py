"""CPU tests of the per-cell accounting behind bench.py's roofline objects
(the algorithmic bytes and flops of the dominant kernels, TENO5 and TENO6
Euler): TENO5 m = 14 unknowns, N_s = 30 large-stencil cells; TENO6 m = 20,
N_s = 42; 3 directional stencils of 12 cells with 5 unknowns, N_q = 3 Gauss
points per edge."""
import bench


def test_reconstruction_bytes():
    # E = m N_s + 3*12*5 matrix entries, (N_s + 36) int32 stencil ids, 3 x 4
    # FP64 states (U^(s), U^n read, U^(s+1) written), geometry 1/|V| + 3 face
    # ids + 1.5 faces x (3 doubles + 2 int32 + 2 int8), 4 selection bytes and
    # the stencil mask
    geo = 8 + 12 + 1.5 * 34
    e5 = 14 * 30 + 3 * 12 * 5
    assert bench.algorithmic_bytes(5, 4, "fp64_native") == e5 * 8 + 66 * 4 + 96 + geo + 5
    assert bench.algorithmic_bytes(5, 4, "fp64_pairs") == bench.algorithmic_bytes(5, 4, "fp64_native")
    assert bench.algorithmic_bytes(5, 4, "fp32_mixed") == e5 * 4 + 66 * 4 + 96 + geo + 5
    # the hot-path table's per-cell-stage figures: ~5.3 KB / 2.9 KB (TENO5),
    # ~8.7 KB / 4.6 KB (TENO6)
    assert abs(bench.algorithmic_bytes(5, 4, "fp64_pairs") - 5300) < 100
    assert abs(bench.algorithmic_bytes(5, 4, "fp32_mixed") - 2900) < 100
    e6 = 20 * 42 + 180
    assert bench.algorithmic_bytes(6, 4, "fp64_pairs") == e6 * 8 + 78 * 4 + 96 + geo + 5
    assert abs(bench.algorithmic_bytes(6, 4, "fp64_pairs") - 8700) < 150
    assert abs(bench.algorithmic_bytes(6, 4, "fp32_mixed") - 4600) < 150


def test_vjp_bytes():
    # W pairs N_s x 3N_q x 8, halo positions N_s x 2, Uq_bar 3N_q x 4 x 8,
    # selection bytes 4, the dU_0 term 4 x 8
    assert bench.algorithmic_vjp_bytes(5, 3) == 30 * 9 * 8 + 60 + 9 * 32 + 4 + 32 == 2544


def test_native_flops():
    # W form, per variable: (N_s + 36) differences, N_s x 3N_q multiply-adds
    # for U_0 + W d, 3N_q additions; TENO5 N_s = 30, TENO6 N_s = 42
    assert bench.algorithmic_fp64_flops(5, 4, 3) == 4 * (66 + 2 * 30 * 9 + 9) == 4 * 615
    assert bench.algorithmic_fp64_flops(6, 4, 3) == 4 * (78 + 2 * 42 * 9 + 9) == 4 * 843


def test_traffic_table_keyed_by_kernel_source():
    h = bench.kernels_hash()
    saved = dict(bench.NCU_TRAFFIC_PER_CELL)
    try:
        bench.NCU_TRAFFIC_PER_CELL[("fp64_pairs", 6)] = (100.0, h)
        bench.NCU_TRAFFIC_PER_CELL[("fp32_mixed", 6)] = (50.0, "0" * 16)  # another build
        assert bench.ncu_traffic("fp64_pairs", 6, 3) == 300.0
        assert bench.ncu_traffic("fp32_mixed", 6, 3) is None
        assert bench.ncu_traffic("fp64_pairs", 7, 1) is None
    finally:
        bench.NCU_TRAFFIC_PER_CELL.clear()
        bench.NCU_TRAFFIC_PER_CELL.update(saved)
