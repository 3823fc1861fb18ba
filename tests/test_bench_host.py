"""Host arithmetic of bench.py, without a GPU: the matrix-element flop model,
the update-tile count behind the inverse's FP64-equivalent rate, and the
roofline record, including the DRAM traffic it reads from the ncu summaries
under profiles/ for each kernel group that can dominate a step."""
import types

import numpy as np
import pytest

import bench
from paper_1111_4429_gb300 import synth


def _shape(name):
    p = synth.CONFIGS[name]
    bvec, _ = synth.cubic_cell(p["a"])
    geps = synth.gsphere(bvec, (0.1, 0.0, 0.0), p["ecut_eps"])
    return types.SimpleNamespace(fft=p["fft"], geps=geps, ng=geps.shape[0], nv=p["nv"], nc=p["nc"],
                                 npairs=p["nv"] * p["nc"])


def test_epsilon_spheres_of_the_two_cells():
    assert _shape("c1").ng == 2120
    assert _shape("c2").ng == 7180


@pytest.mark.parametrize("name,per_pair", [("c1", 3.08e6), ("c2", 11.35e6)])
def test_mtxel_flops_per_pair(name, per_pair):
    # 5 n log2 n per line over n^2 y lines, (2 g_x + 1) n x lines and
    # (2 g_x + 1)(2 g_y + 1) z lines, plus 6 n^3 for the product: 40^3 with
    # |G_x|, |G_y| <= 8, 7 and 60^3 with 12, 11
    s = _shape(name)
    total, pp = bench.mtxel_flops(s)
    assert abs(pp / per_pair - 1.0) < 2e-3
    assert total > s.npairs * pp


def test_update_tiles_sum_to_the_sweep_work():
    # every step's look-ahead and bulk tiles, 32 complex multiply-adds of 8
    # flop per element of a 128 x 32 tile, add up to the sweep's 4 N_G^3 plus
    # the padding of the diagonal tiles, which shrinks as N_G grows
    ratios = []
    for ng in (2120, 7180):
        tiles = sum(sum(bench.oz_tiles(ng, k0)) for k0 in range(0, ng, 32))
        ratios.append(tiles * 8.0 * 128 * 32 * 32 / (4.0 * ng ** 3))
    assert 1.0 <= ratios[1] < ratios[0] < 1.15


def _kt(dominant):
    kt = {"band_transform": (12, 3.6), "pair_yxpass": (18, 20.0), "pair_zgather": (18, 15.0),
          "chi_split": (6, 11.0), "chi_tc": (6, 20.0), "chi_reduce": (6, 2.0), "oz_update": (225, 20.0),
          "oz_update_ahead": (224, 8.0), "inverse": (1, 63.0)}
    n, _ = kt[dominant]
    kt[dominant] = (n, 150.0)
    return kt


@pytest.mark.parametrize("size", ["c1", "c2"])
@pytest.mark.parametrize("dominant,bound", [("pair_yxpass", "alu"), ("chi_tc", "tensor"), ("oz_update", "tensor")])
def test_roofline_record(size, dominant, bound):
    s = _shape(size)
    peaks = {"hbm_gbs": 6775.6, "bf16_tflops": 1939.0, "bf16_tflops_sustained": 1737.8}
    kt = _kt(dominant)
    step = 375.0
    roof = bench._roofline(s, kt, step, peaks, "measured", size_tag=size)
    assert roof["bound"] == bound
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    assert 0.0 < roof["frac"] < 1.5
    assert roof["share_of_step"] == pytest.approx(150.0 / step)
    assert roof["launches_per_step"] == kt[dominant][0]
    # every group that can dominate has a current DRAM count in profiles/
    assert roof["traffic"] is not None and roof["traffic"] > 0
    if dominant == "oz_update":
        assert roof["fp64_equivalent_tflops"] > 0 and roof["peak"] == peaks["bf16_tflops_sustained"]
    if dominant == "pair_yxpass":
        flops = bench.mtxel_flops(s)[0]
        expect = flops / ((150.0 + 15.0 + 3.6) / 1e3) / 1e12
        assert roof["achieved"] == pytest.approx(expect)
        assert roof["peak"] == pytest.approx(bench.FP32_PEAK_TFLOPS)


def test_traffic_records_are_unique():
    # one record per tag, so an edited summary cannot leave a stale twin
    import glob
    import os
    import re
    seen = {}
    for path in glob.glob(os.path.join(os.path.dirname(bench.__file__), "profiles", "*.md")):
        for tag in re.findall(r"traffic\[([A-Za-z0-9_]+)\]:", open(path).read()):
            assert tag not in seen, (tag, path, seen.get(tag))
            seen[tag] = path
    for tag in ("pair_yxpass_c1", "pair_yxpass_c2", "chi_tc_c1", "chi_tc_c2", "oz_update_c1", "oz_update_c2"):
        assert tag in seen, tag
