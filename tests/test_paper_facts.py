"""Consistency of the numbers the paper prints (tests/golden/paper_facts.json)."""
import json
import os


def _facts(root):
    return json.load(open(os.path.join(root, "tests", "golden", "paper_facts.json")))


def test_water_basis_size(repo_root):
    f = _facts(repo_root)["water_basis"]
    assert f["molecules"] * f["functions_per_molecule"] == f["total_functions"]


def test_apparent_throughput_fraction_of_peak(repo_root):
    f = _facts(repo_root)["node_peak"]
    peak = f["cores"] * f["ghz"] * f["dp_flop_per_cycle_avx"]
    assert abs(peak - 332.8) < 1e-9
    assert round(100 * f["apparent_gflops_1node"] / peak) == f["fraction_of_peak_percent"]
