"""The measurement arithmetic of bench.py (CPU only): algorithmic bytes and flops per DOF,
the n_0.8 interpolation, the FP64 peak derivation and the ncu-summary parser.

The byte and flop counts are checked against their closed forms written out independently
here (Sec. 2: n = E N^3; one PCG iteration reads p once, writes w once, streams six factor
words and one int32 index per local node, and moves 13 vector words per unique DOF).
"""
import math
import os

import pytest

import bench


@pytest.mark.parametrize("N", [3, 5, 7, 9, 11, 15])
def test_bp5_units_closed_form(N):
    p1 = N + 1
    local_per_dof = p1 ** 3 / N ** 3
    elem_bytes, iter_bytes, flops = bench.bp5_units(N)
    assert elem_bytes == pytest.approx(16 + 52 * local_per_dof)
    assert iter_bytes == pytest.approx(104 + 52 * local_per_dof)
    # the element work of the factored stiffness: 6 contractions of length p1 per node (12 p1 flops)
    # plus the 15-flop application of the symmetric 3x3 factor, per local node
    assert flops == pytest.approx((12 * p1 + 15) * local_per_dof)


def test_bp5_units_n7_values():
    elem_bytes, iter_bytes, flops = bench.bp5_units(7)
    assert round(iter_bytes, 1) == 181.6
    assert round(elem_bytes, 1) == 93.6
    assert round(flops, 1) == 165.7


def test_recompute_units_fewer_bytes_more_flops():
    for N in (3, 7, 11):
        e0, i0, f0 = bench.bp5_units(N)
        e1, i1, f1 = bench.bp5_units_recompute(N)
        assert e1 < e0 and i1 < i0 and f1 > f0
        p1 = N + 1
        assert e0 - e1 == pytest.approx(24 * p1 ** 3 / N ** 3)


def test_n08_interpolates_log_linearly():
    ns = [1e4, 1e5, 1e6, 1e7]
    rates = [1.0, 4.0, 9.0, 10.0]  # r_max = 10, target 8 lies between 1e5 (4) and 1e6 (9)
    n80 = bench.n_08(ns, rates)
    t = (8.0 - 4.0) / (9.0 - 4.0)
    assert n80 == pytest.approx(math.exp(math.log(1e5) + t * (math.log(1e6) - math.log(1e5))))
    assert bench.n_08([1e4, 1e5], [9.0, 10.0]) == 1e4  # first sample already above 80 %


def test_fp64_peak_from_unit_counts():
    tf, src = bench.fp64_peak_tflops({"sm_max_mhz": 2070.0})
    assert tf == pytest.approx(2 * 2 * 152 * 2070e6 / 1e12, rel=1e-3)


def test_max_over_ranks_single_rank():
    assert bench.max_over_ranks(3.5, 1, None, None) == 3.5


def test_ncu_traffic_reads_committed_profiles():
    for name in os.listdir(os.path.join(bench.ROOT, "profiles")):
        if name.startswith("bk5_"):
            v = bench.ncu_traffic(name)
            assert v is not None and 1e9 < v < 2e10, name
    assert bench.ncu_traffic("no_such_profile.md") is None


def test_ncu_value_reads_instruction_counts(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "x.md").write_text("# t\n\ndfma_per_element: 12288\ndadd_per_element: 3.5e3\nother: z\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_value("x.md", "dfma_per_element") == 12288.0
    assert bench.ncu_value("x.md", "dadd_per_element") == 3500.0
    assert bench.ncu_value("x.md", "other") is None
    assert bench.ncu_value("missing.md", "dfma_per_element") is None


def test_bk_flop_counts_per_dof():
    """Work per DOF of the element operators: BK5 12 p1^4 + 15 p1^3 per element (Eq. (22)),
    BK3 the interpolate-then-differentiate count of Eqs. (31)-(33), BK1 the mass J^T B J (Eq. (34));
    N = 7 gives 165.7, 443.6 and 184.3 flops per DOF."""
    per_dof = {bp: bench.bk_flops(bp, 7) / 7 ** 3 for bp in (1, 3, 5)}
    assert abs(per_dof[5] - 165.7) < 0.05
    assert abs(per_dof[3] - 443.6) < 0.05
    assert abs(per_dof[1] - 184.3) < 0.05
    assert bench.bk_flops(6, 7) == bench.bk_flops(5, 7) and bench.bk_flops(4, 3) == bench.bk_flops(3, 3)
