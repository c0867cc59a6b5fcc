"""Host logic of bench.py's JSON line (no GPU): the SA sketch's figures nested
inside the roofline object."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_sa_sketch_nested_in_roofline():
    roof = {"kernel": "k_lsqr_pass", "bound": "hbm", "achieved": 5371.1, "peak": 6668.9, "unit": "GB/s",
            "frac": 0.805, "peak_source": "measured", "alg_bytes_per_launch": 2348810244, "traffic": 2.2983e9}
    sk = {"call": "cw_sketch_csr", "bound": "hbm", "achieved": 1893.7, "peak": 6668.9, "unit": "GB/s",
          "frac": 0.284, "peak_source": "measured", "alg_bytes_per_call": 2349072388, "ms": 1.2405,
          "nnz_per_s": 2.16e11, "traffic": 2.3773e9, "traffic_of": "k_apply_csr", "stages_ms": {"k_apply_csr": 0.64},
          "segment_read_rates": {"random_64B_GBps": 2662.2, "sequential_64B_GBps": 6241.5},
          "apply_gather_GBps": 3332.1, "apply_frac_of_random_64B": 1.25}
    out = bench.with_sa_sketch(roof, sk)
    for k, v in roof.items():
        assert out[k] == v
    sa = out["sa_sketch"]
    assert sa["frac"] == 0.284 and sa["ms"] == 1.2405 and sa["call"] == "cw_sketch_csr"
    assert sa["segment_read_rates"]["random_64B_GBps"] == 2662.2
    assert sa["apply_frac_of_random_64B"] == 1.25
    assert "stages_ms" not in sa and "sa_sketch" not in roof   # compact, and the input is not modified
    json.dumps(out)


def test_sa_sketch_passthrough_without_figures():
    assert bench.with_sa_sketch(None, {"frac": 0.3}) is None
    roof = {"kernel": "k_lsqr_pass", "frac": 0.8}
    assert bench.with_sa_sketch(roof, None) == roof
    assert bench.with_sa_sketch(roof, {}) == roof
    partial = bench.with_sa_sketch(roof, {"frac": 0.3, "ms": 1.3})
    assert partial["sa_sketch"] == {"frac": 0.3, "ms": 1.3}
