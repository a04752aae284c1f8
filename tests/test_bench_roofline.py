"""bench.py's roofline arithmetic (CPU): the algorithmic bytes and flops each kernel
class is charged with, the choice of the dominant class and the fraction of peak."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_class_amounts():
    import bench
    m, n, l = 512, 65536, 2048
    assert bench.class_amount(5, m, n, l, 10) == (10 * 8.0 * m * n, "GB/s", "hbm")      # one pass per iteration
    assert bench.class_amount(0, m, n, l, 3)[0] == 3 * 8.0 * m * n
    assert bench.class_amount(2, m, n, l, 1) == (2 * 16.0 * m * n, "GB/s", "alu")      # two fixed-point passes
    qr = bench.class_amount(3, m, n, l, 1)
    assert qr[1:] == ("TFLOP/s", "alu")                                                 # l <= 2048: FP64
    assert qr[0] == pytest.approx(8.0 * m * m * (l - m / 3.0))                          # Householder QR of Y
    assert bench.class_amount(7, m, n, l, 1) == (8.0 * m ** 3 / 6.0, "TFLOP/s", "alu")  # P R^-1
    assert bench.class_amount(4, m, n, l, 1)[0] == 8.0 * m * n + 16.0 * l * m          # read A, write Y
    # a tall sketch: the blocked QR on the tensor cores, then the triangle's pivoted QR (FP64)
    m, n, l = 2048, 262144, 8192
    qr = bench.class_amount(3, m, n, l, 2)
    assert qr == (2 * 8.0 * m * m * (l - m / 3.0), "TFLOP/s", "tensor")
    assert bench.class_amount(6, m, n, l, 1) == (16.0 * m ** 3 / 3.0, "TFLOP/s", "alu")


def test_side_roofline_picks_the_dominant_class():
    import bench
    shapes = [(512, 65536)]
    times = {0: (0, 0.0), 1: (0, 0.0), 2: (10, 5.0), 3: (1, 12.0), 4: (1, 2.0), 5: (60, 3.5), 6: (0, 0.0),
             7: (1, 1.0)}
    pk = {"hbm_gbs": 6690.5}
    r = bench.side_roofline(shapes, lambda i, k: times[k], pk)
    assert r["kernel"] == "pivoted_qr"
    flops = 8.0 * 512 ** 2 * (2048 - 512 / 3.0)
    assert r["achieved"] == pytest.approx(flops / 0.012 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / bench.FP64_NOMINAL_TFLOPS)
    assert r["ms_by_class"]["cg_fused"] == 3.5
    # a tall sketch whose blocked QR dominates: the tensor-core bound with the FP64-equivalent peak
    times = {k: (0, 0.0) for k in bench.KERNEL_CLASSES}
    times[3] = (1, 50.0)
    times[6] = (1, 40.0)
    r = bench.side_roofline([(2048, 262144)], lambda i, k: times[k], {"hbm_gbs": 6690.5, "bf16_tflops": 1925.0})
    assert r["kernel"] == "pivoted_qr" and r["bound"] == "tensor"
    assert r["peak"] == pytest.approx(1925.0 / bench.OZAKI_MEAN_PAIRS)
    assert r["achieved"] == pytest.approx(8.0 * 2048 ** 2 * (8192 - 2048 / 3.0) / 0.05 / 1e12)


def test_aggregate_and_batch_cost():
    import bench
    assert bench.aggregate_value(4, 10, 2000.0) == pytest.approx(20.0)    # 40 solves in 2 s
    assert bench.batch_cost(2, 10) == 8 + 40


def test_cg_pass_time_counts_iterations_not_launches():
    import bench
    empty = {k: (0, 0.0) for k in range(8)}
    # two passes: 48 launches of each product for 39 iterations (9 returned at once after the test fired)
    st = {**empty, 0: (48, 24.2), 1: (48, 24.8)}
    assert bench.cg_pass_time(st, 39) == (pytest.approx((24.2 + 24.8) / 78), 2)
    # one pass (class 0 alone): 48 launches for 39 iterations
    st = {**empty, 0: (48, 41.3)}
    assert bench.cg_pass_time(st, 39) == (pytest.approx(41.3 / 39), 1)
    # the fused solve (class 5 counts its iterations)
    st = {**empty, 5: (61, 3.5)}
    assert bench.cg_pass_time(st, 61) == (pytest.approx(3.5 / 61), 1)
    # no CG run: no time
    assert bench.cg_pass_time(empty, 0) == (0.0, 2)
