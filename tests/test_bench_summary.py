"""The compact summary that closes the benchmark's JSON line (host logic, no GPU): it carries the
variant times and HBM fractions and the serving comparison, rounded, and stays short enough to
survive in the last 1.5 KB of the line."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line():
    variants = {f"variant_{k}": {"kernel": "k" * 80, "ms_per_step": 0.5 + k / 7.0, "mlups": 1e4,
                                 "hbm_frac": 0.5 + k / 100.0} for k in range(10)}
    variants["missing"] = None
    side = {"solves_per_s": 13.861234, "latency_p50_s": 1.2151, "latency_p99_s": 54.6213}
    plain = {"solves_per_s": 12.5111, "latency_p50_s": 35.3321, "latency_p99_s": 61.3631}
    serving = {"requests": 2000, "batched": side, "sequential_fp32": plain,
               "sustained": {"arrival_rate_per_s": 10.0087, "batched": side, "sequential_fp32": plain},
               "errors_vs_fp64": {"x": "y" * 5000}}
    return {"metric": "rD3Q53 MLUPS", "value": 15000.0, "variants": variants, "serving": serving}


def test_summary_content():
    s = bench._summary(_line())
    assert set(s["variants_ms_per_step"]) == {f"variant_{k}" for k in range(10)}
    assert s["variants_ms_per_step"]["variant_7"] == round(0.5 + 1.0, 4)
    assert s["variants_hbm_frac"]["variant_3"] == 0.53
    sv = s["serving"]
    assert sv["requests"] == 2000
    assert sv["solves_per_s"] == [13.861, 12.511]
    assert sv["p50_s"] == [1.215, 35.332] and sv["p99_s"] == [54.621, 61.363]
    assert sv["sustained"]["arrival_rate_per_s"] == 10.009


def test_summary_is_short_and_optional():
    assert len(json.dumps(bench._summary(_line()))) < 1400
    assert bench._summary({"metric": "m", "value": 1.0}) == {"variants_ms_per_step": {}, "variants_hbm_frac": {}}
