"""Host logic of the bench's roofline record: the dominant solver operation is chosen with
its storage variants merged (the FP64 colour sweep in the plain and the colour-split
storage is one operation), the field has its own record, and the work counts only the
launches' recorded units."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_roof", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def rec(ms, launches, bytes_, flops):
    return {"ms": ms, "launches": launches, "timed": launches, "bytes": bytes_, "flops": flops}


def test_colour_sweep_storages_are_one_operation(bench):
    prof = {
        "field_df32": rec(413.0, 40, 1e9, 4e12),
        "rbgs_split_f64@129": rec(312.7, 400, 400 * 4.6e8, 400 * 1.07e8),
        "rbgs_f64@65": rec(270.0, 960, 960 * 5.7e7, 960 * 1.3e7),
        "solve_cta_f64@33": rec(220.0, 5, 0.0, 0.0),
    }
    roof = bench.roofline(prof, {"hbm_gbs": 6785.9})
    assert roof["kernel"] == "rbgs_split_f64@129"
    assert roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    # 1.07e8 flop per launch over 312.7 ms / 400 launches
    assert roof["achieved"] == pytest.approx(1.07e8 / (312.7e-3 / 400) / 1e12)
    assert roof["operation_share_of_profiled_time"] == pytest.approx((312.7 + 270.0) / (413 + 312.7 + 270 + 220))
    field = bench.field_roofline(prof)
    assert field["kernel"] == "field_df32" and field["node_features_per_s"] == pytest.approx(1e12 / 0.413)


def test_fp32_classes_use_hbm_bound(bench):
    prof = {"rbgs_split_f32@257": rec(65.7, 10, 10 * 2.65e8, 10 * 6.1e8),
            "cg_apply_dot": rec(40.0, 10, 10 * 1.2e9, 10 * 2.7e8)}
    roof = bench.roofline(prof, {"hbm_gbs": 6785.9}, lambda k: k.startswith("rbgs"))
    assert roof["kernel"] == "rbgs_split_f32@257" and roof["bound"] == "hbm"
    assert roof["achieved"] == pytest.approx(2.65e8 / 6.57e-3 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / 6785.9)


def test_tensor_core_field_record(bench):
    """With the tensor-core field, its record counts 112 bf16 flops per node-feature of the
    field_tc launches against the measured sustained bf16 rate; the node-features per second
    cover every field launch (the x = n - 1 column runs in double-float); xslices is field
    work, not a solver operation."""
    prof = {"field_tc": rec(100.0, 40, 1e9, 4e12), "field_df32": rec(5.0, 40, 1e7, 4e10),
            "xslices": rec(1.0, 40, 1e6, 1e6), "rbgs_split_f64@129": rec(312.7, 400, 400 * 4.6e8, 400 * 1.07e8)}
    peaks = {"hbm_gbs": 6785.9, "bf16_tflops": 1949.3, "bf16_tflops_sustained": 1708.4}
    field = bench.field_roofline(prof, peaks)
    assert field["kernel"] == "field_tc" and field["unit"] == "TFLOP/s"
    assert field["achieved"] == pytest.approx(112 * 1e12 / 0.1 / 1e12)
    assert field["frac"] == pytest.approx(field["achieved"] / 1708.4)
    assert field["node_features_per_s"] == pytest.approx((1e12 + 1e10) / 0.106)
    assert bench.roofline(prof, peaks)["kernel"] == "rbgs_split_f64@129"
    assert not bench.solver_class("xslices")
