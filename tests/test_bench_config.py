"""Host logic of bench.py's AIR configuration (no GPU): the coarsest level per
workload and its record in the JSON line's config."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class Args:
    config = "hex32_s4"
    max_coarse = None
    coarse_sweeps = None
    theta, phi_R, phi_A, distance, nair = 0.5, 0.0, 0.05, 1, 0
    concurrent, timing_every, precision, si_fixed = 1, 9, 1, None


def test_coarsest_level_per_workload():
    a = Args()
    assert bench.coarsest(a) == (40000, 3)
    for name in ("hex64_s8", "tet40_s8"):
        assert bench.coarsest(a, name) == (40000, 3)
    for name in ("hex8_s2", "hex24_s4_adj", "tet16_s8"):   # small meshes: the library's
        assert bench.coarsest(a, name) == (100, 20)
    a.max_coarse, a.coarse_sweeps = 500, 4                  # the flags override the table
    assert bench.coarsest(a, "hex8_s2") == (500, 4)


def test_air_settings_follow_the_workload_and_the_record_matches():
    a = Args()
    kw = bench.air_settings(a, 2, "tet40_s8")
    assert kw["distance"] == 2 and (kw["max_coarse"], kw["coarse_sweeps"]) == (40000, 3)
    assert bench.air_settings(a)["distance"] == 1
    rec = bench.bench_config(a, 1)["air"]
    assert (rec["max_coarse"], rec["coarse_sweeps"]) == bench.coarsest(a)
    assert rec["theta"] == a.theta and rec["phi_A"] == a.phi_A
