"""The bench's roofline arithmetic: algorithmic flops and bytes per launch of each kernel
class, checked against counts written out by hand for the 2D 255^2 x 256 workload
(16,646,400 unknowns), and the structure of the recorded ncu traffic."""
import json
import os

import bench

U = 255 * 255 * 256


def test_time_kernel_counts():
    # four real transforms of length 256 at 2.5 n log2 n each per real sequence
    # (10 log2 n = 80 per unknown), two spectral multiplies (6), three scalings (3)
    assert bench.algorithmic_flops("time_f64", 2, 255, 256, U) == 89 * U
    # FP64 vectors in and out (16 B) plus the FP64 spectral table: (n/2+1) x pairs x 2 x 16 B
    table = 129 * ((255 * 255 + 1) // 2) * 2 * 16
    assert bench.algorithmic_bytes("time_f64", 2, 255, 256, U, 8) == 16 * U + table
    # complex64 table for the FP32 kernel
    assert bench.algorithmic_bytes("time_f32", 2, 255, 256, U, 8) == 16 * U + table // 2


def test_dst_and_operator_counts():
    assert bench.algorithmic_flops("dst_x_f64", 2, 255, 256, U) == 2.5 * 8 * U   # log2(256) = 8
    assert bench.algorithmic_bytes("dst_x_f64", 2, 255, 256, U, 8) == 16 * U
    # DST basis: Lambda (v_i + v_{i-2}) - 2 v_{i-1} = 4 flops, + 2 for the fused dot
    assert bench.algorithmic_flops("yt_dot", 2, 255, 256, U) == 6 * U
    # physical residual check: stencil 2d + 2, time band 3, residual and square 3
    assert bench.algorithmic_flops("yt_res", 2, 255, 256, U) == (2 * 2 + 5 + 3) * U
    # variable coefficient: 6d + 1 per L application, time band 3, fused dot 2
    assert bench.algorithmic_flops("yt_dot", 2, 255, 256, U, varcoef=True) == (6 * 2 + 3 + 2) * U
    assert bench.algorithmic_flops("wx_res", 2, 255, 256, U) == 14 * U
    assert bench.algorithmic_bytes("wx_res", 2, 255, 256, U, 8) == 56 * U
    assert bench.algorithmic_flops("yt_resvec", 2, 255, 256, U) == 7 * U
    assert bench.algorithmic_bytes("yt_resvec", 2, 255, 256, U, 8) == 24 * U


def test_double_word_flop_factor():
    # sloppy double-word add 11 FP32 flops, FMA-based product 10, FFT mix 60/40
    assert abs(bench.DW_FP32_FLOPS_PER_FLOP - 10.6) < 1e-12


def test_traffic_records_name_existing_sources():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    with open(os.path.join(root, "profiles", "traffic.json")) as fh:
        rec = json.load(fh)
    for cls, r in rec.items():
        # a record whose sources changed since the capture is reported as null by the
        # bench, so only the structure is checked here
        for f in r["sources"]:
            assert os.path.exists(os.path.join(root, "paper_2306_03574_gb300", "csrc", f)), (cls, f)
        assert len(r["source_hash"]) == 16, cls
        assert r["bytes_per_launch"] == r["dram_read"] + r["dram_write"], cls
        assert os.path.exists(os.path.join(root, r["capture"])), cls
