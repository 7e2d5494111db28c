"""bench.py's algorithmic model (CPU only): the per-launch byte and FMA counts the roofline
divides by, checked against the formulas written out here, and the reported host fields."""
import types

import numpy as np

import bench

ESD = types.SimpleNamespace(PLAIN=0, DEFLATION=1, SUBSPACE_CORRECTION=2)


def _problem(n, nnz):
    return types.SimpleNamespace(n=n, nnz=nnz)


def test_pad_m_matches_the_compiled_column_counts():
    assert [bench.pad_m(m) for m in (0, 1, 8, 9, 16, 17, 24, 25, 32, 33, 64)] == [0, 8, 8, 16, 16, 24, 24, 32, 32, 64, 64]


def test_spmv_model_fp64_and_fp32():
    n, nnz, m = 2_097_152, 14_581_760, 16
    p = _problem(n, nnz)
    lv = (np.array([n // 8]), None, None)
    a64 = types.SimpleNamespace(precision="fp64", m=m)
    by, fm = bench.kernel_model("spmv_pq", p, a64, ESD.DEFLATION, ESD, lv)
    assert by == 12 * nnz + 20 * n + 8 * m * n  # A (value + column), p read, q written, AW
    assert fm == nnz + n  # (AW)^T p runs in double-float on the FP32 pipe for m <= 32
    by, fm = bench.kernel_model("spmv_pq", p, a64, ESD.PLAIN, ESD, lv)
    assert (by, fm) == (12 * nnz + 20 * n, nnz + n)
    a64w = types.SimpleNamespace(precision="fp64", m=40)  # padded to 64: FP64 W terms
    by, fm = bench.kernel_model("spmv_pq", p, a64w, ESD.DEFLATION, ESD, lv)
    assert fm == nnz + n + 40 * n
    a32 = types.SimpleNamespace(precision="fp32", m=m)
    by, fm = bench.kernel_model("spmv_pq", p, a32, ESD.DEFLATION, ESD, lv)
    assert by == 8 * nnz + 12 * n + 4 * n + 4 * m * n  # FP32 pairs, s = A 1 read, FP32 AW
    assert fm == nnz + n + m * n


def test_spmv_model_column_free_copy():
    n, nnz = 2_097_152, 14_581_760
    p = _problem(n, nnz)
    lv = (np.array([n // 8]), None, None)
    a32 = types.SimpleNamespace(precision="fp32", m=16)
    slices, slots_a = n // 32, 7 * n
    lay = {"column_free": [True, True, True], "slot_entries": [slots_a, 3 * n, 3 * n], "slices": slices}
    by, fm = bench.kernel_model("spmv_pq", p, a32, ESD.PLAIN, ESD, lv, lay)
    # 4-byte slot values and 32 bytes of slot bases per slice instead of 8-byte pairs
    assert by == 4 * slots_a + 32 * slices + 12 * n + 4 * n
    assert fm == nnz + n
    # the deflated FP32 product keeps the pairs whatever the layout
    by, _ = bench.kernel_model("spmv_pq", p, a32, ESD.DEFLATION, ESD, lv, lay)
    assert by == 8 * nnz + 12 * n + 4 * n + 4 * 16 * n
    # without the copy, or in FP64, the pairs
    no = {"column_free": [False] * 3, "slot_entries": [0] * 3, "slices": slices}
    assert bench.matrix_bytes(p, 4, no, 0) == 8 * nnz
    assert bench.matrix_bytes(p, 8, lay, 0) == 12 * nnz
    assert bench.matrix_bytes(p, 4, lay, 1) == 4 * 3 * n + 32 * slices


def test_update_model():
    n, m = 1000, 16
    p = _problem(n, 7 * n)
    n0 = 125
    lv = (np.array([n0]), None, None)
    a = types.SimpleNamespace(precision="fp64", m=m)
    by, fm = bench.kernel_model("update", p, a, ESD.DEFLATION, ESD, lv)
    assert by == 16 * n + 32 * n + 8 * m * n + 16 * n0
    assert fm == 3 * n + 2 * n0  # AW y in double-float
    by, fm = bench.kernel_model("update", p, a, ESD.PLAIN, ESD, lv)
    assert (by, fm) == (16 * n + 32 * n + 16 * n0, 3 * n + 2 * n0)


def test_gamma_model_is_the_papers_ratio():
    """Eq. ganma for the 128^3 7-point workload with m = 16: (116 + 16 m + 24 nnz_av) /
    (100 + 24 nnz_av) = 2.02."""
    nnz_av = 14_581_760 / 2_097_152
    g = (116 + 16 * 16 + 24 * nnz_av) / (100 + 24 * nnz_av)
    assert abs(g - 2.02) < 0.005


def test_host_info_fields():
    h = bench.host_info()
    assert h["nproc"] >= 1 and isinstance(h["cpu_model"], str) and h["machine"]


def test_pair_models_share_the_matrix_once():
    """The paired launches: the matrix (and s = A 1, 1/l_ii) once, each system's vectors."""
    n, nnz = 2_097_152, 14_581_760
    p = _problem(n, nnz)
    n0 = n // 8
    lv = (np.array([n0]), None, None)
    a32 = types.SimpleNamespace(precision="fp32", m=16)
    slices, slots_a = n // 32, 7 * n
    lay = {"column_free": [True, True, True], "slot_entries": [slots_a, 3 * n, 3 * n], "slices": slices}
    by, fm = bench.kernel_model("spmv_pq", p, a32, ESD.PLAIN, ESD, lv, lay, pair=True)
    # slots and bases, s = A 1 once; p read, q written and the 4 n term per system
    assert by == 4 * slots_a + 32 * slices + 4 * n + 2 * 12 * n
    assert fm == 2 * (nnz + n)
    by, fm = bench.kernel_model("update", p, a32, ESD.PLAIN, ESD, lv, lay, pair=True)
    # per system: x read and written in FP64, p, q, r read, r written, y written on level 0;
    # 1/l_ii of level 0 once
    assert by == 2 * (16 * n + 16 * n + 4 * n0) + 4 * n0
    assert fm == 2 * (3 * n + 2 * n0)


def test_pair_launch_count():
    """esd_solve_pair's graph: 2 residuals, the loop condition and 2 final kernels; per
    refinement step both systems' prep, start (residual, update, 3 + 3 sweeps), finish and
    residual, the pack and unpack of p and four loop conditions; one body (SpMV, update,
    3 + 3 sweeps) per paired iteration and per iteration a system ran alone."""
    info = {"fwd_levels": 4, "bwd_levels": 4}
    start, body = 1 + 1 + 3 + 3, 2 + 3 + 3
    per_step = 2 * (1 + start + 1 + 1) + 2 + 4
    # 9 steps for the longer system, 1500 + 1400 iterations of which 1300 paired
    assert bench.pair_launch_count(info, [1500, 1400], [9, 8], 1300) == 5 + 9 * per_step + body * (2900 - 1300)
    # nothing paired: every iteration runs alone
    assert bench.pair_launch_count(info, [10, 0], [1, 0], 0) == 5 + per_step + body * 10
