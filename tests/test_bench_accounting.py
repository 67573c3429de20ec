"""CPU tests of the per-cell accounting behind bench.py's roofline objects
(the algorithmic bytes and flops of the dominant kernels, TENO5 Euler):
m = 14 unknowns, N_s = 30 large-stencil cells, 3 directional stencils of 12
cells with 5 unknowns, N_q = 3 Gauss points per edge."""
import bench


def test_reconstruction_bytes():
    # E = m N_s + 3*12*5 = 600 matrix entries, (N_s + 36) int32 stencil ids,
    # 4 FP64 states, 1 stencil mask byte, 4 selection bytes
    e = 14 * 30 + 3 * 12 * 5
    assert bench.algorithmic_bytes(5, 4, "fp64") == e * 8 + 66 * 4 + 32 + 1 + 4 == 5101
    assert bench.algorithmic_bytes(5, 4, "fp32_mixed") == e * 4 + 66 * 4 + 32 + 1 + 4 == 2701


def test_vjp_bytes():
    # W pairs N_s x 3N_q x 8, halo positions N_s x 2, Uq_bar 3N_q x 4 x 8,
    # selection bytes 4, the dU_0 term 4 x 8
    assert bench.algorithmic_vjp_bytes(5, 3) == 30 * 9 * 8 + 60 + 9 * 32 + 4 + 32 == 2544


def test_native_flops():
    # per variable: (N_s + 36) differences, 2E matvec, 2(m + 15) beta, 25 for
    # the selection, 2 * 3N_q * m evaluation products and 3N_q sums
    per_var = 66 + 2 * 600 + 2 * 29 + 25 + 2 * 9 * 14 + 9
    assert per_var == 1610
    assert bench.algorithmic_fp64_flops(5, 4, 3) == 4 * per_var


def test_traffic_table_scales_by_cells():
    assert bench.ncu_traffic("fp64", 5, 2) == 2 * bench.NCU_TRAFFIC_PER_CELL[("fp64", 5)]
    assert bench.ncu_traffic("fp64", 7, 1) is None
