"""Host logic of the benchmark line, checked on the CPU: the work model's node
counts against the library's dimension tree, and the roofline object's choice
of the dominant kernel family and its arithmetic (achieved = work per launch /
time per launch, peak = the unit's figure for the family's bound)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1708_03340_gb300 import htgb  # noqa: E402


@pytest.mark.parametrize("d", [2, 3, 5, 8, 13, 256])
def test_work_model_counts_the_tree_nodes(d):
    """12 K^4 per non-root inner node, n K (K + 2r) per leaf, 9 K^3 per
    non-root node (one Gramian each): the counts come from the balanced tree
    the library builds (Sec. 2), not from a formula in d."""
    tree = htgb.HTTree(d)
    nodes = [tree.node(t) for t in range(tree.nn)]
    leaves = sum(1 for v in nodes if v["son1"] < 0)
    inner_nonroot = sum(1 for v in nodes if v["son1"] >= 0 and v["parent"] >= 0)
    nonroot = sum(1 for v in nodes if v["parent"] >= 0)
    n, K, r = 100, 8, 3
    work, eig = bench.model_flops(d, n, K, r)
    assert leaves == d
    assert work == inner_nonroot * 12.0 * K ** 4 + leaves * n * K * (K + 2 * r)
    assert eig == nonroot * 9.0 * K ** 3


PEAKS = {"bf16_cublas": 2000.0, "hbm_gbs": 8000.0, "fp32_fma": 81.0, "fp64_fma": 1.5}


def _prof(ms):
    """A profile of two steps: family -> (ms, launches, work)."""
    work = {"qr": 4.0e12, "gemm": 8.0e15, "split": 2.0e11, "eig": 3.0e11, "copy": 1.0e9}
    launches = {"qr": 10, "gemm": 40, "split": 20, "eig": 2, "copy": 8}
    return {k: {"ms": ms[k], "launches": launches[k], "flops": work[k]} for k in ms}


def test_roofline_picks_the_family_with_the_most_time():
    prof = _prof({"qr": 120.0, "gemm": 100.0, "split": 90.0, "eig": 30.0, "copy": 500.0})
    top = bench.roofline_of(prof, 2, PEAKS)
    # copy is not one of the four families, however long it takes
    assert set(top["families"]) == {"qr", "gemm", "split", "eig"}
    assert top["kernel"].startswith("qr_df_kernel")
    assert top["ms_per_step"] == pytest.approx(60.0)
    prof["gemm"]["ms"] = 130.0
    assert bench.roofline_of(prof, 2, PEAKS)["kernel"].startswith("oz_gemm_kernel")


def test_roofline_arithmetic_per_family():
    prof = _prof({"qr": 120.0, "gemm": 100.0, "split": 90.0, "eig": 30.0})
    f = bench.roofline_of(prof, 2, PEAKS)["families"]
    # qr: 4e12 flop over 10 launches of 12 ms -> 33.3 TFLOP/s against the FP32
    # instruction rate (flop rate / 2) over 6.75 instructions per flop
    assert f["qr"]["achieved"] == pytest.approx(4.0e12 / 10 / 0.012 / 1e12)
    assert f["qr"]["peak"] == pytest.approx(81.0 / 2 / 6.75)
    assert (f["qr"]["bound"], f["qr"]["unit"]) == ("alu", "TFLOP/s")
    assert f["gemm"]["achieved"] == pytest.approx(8.0e15 / 40 / 0.0025 / 1e12)
    assert (f["gemm"]["bound"], f["gemm"]["peak"]) == ("tensor", 2000.0)
    assert f["split"]["achieved"] == pytest.approx(2.0e11 / 20 / 0.0045 / 1e9)
    assert (f["split"]["bound"], f["split"]["unit"], f["split"]["peak"]) == ("hbm", "GB/s", 8000.0)
    assert (f["eig"]["bound"], f["eig"]["peak"]) == ("alu", 1.5)
    for k, v in f.items():
        assert v["frac"] == pytest.approx(v["achieved"] / v["peak"])
        assert v["work_per_launch"] * v["launches_per_step"] * 2 == pytest.approx(prof[k]["flops"])


def test_roofline_skips_families_without_work():
    prof = _prof({"qr": 120.0, "gemm": 100.0})
    prof["qr"]["flops"] = 0.0
    top = bench.roofline_of(prof, 2, PEAKS)
    assert set(top["families"]) == {"gemm"}
    assert bench.roofline_of({"copy": {"ms": 1.0, "launches": 1, "flops": 1.0}}, 1, PEAKS) is None
