"""The autotuner's cache (no GPU): keys, round trip, and the bench's fallback."""
import json
import os


def test_cache_round_trip(tmp_path):
    from paper_2605_24882_gb300 import autotune
    from wm_workloads import WORKLOADS
    c = WORKLOADS["sphere_p2_j6_mixed_s256"]
    key = autotune.cache_key(c, c["n_samples"], "NVIDIA GB300")
    assert key == "sphere/p2/64x64/L7/s256/mixed/NVIDIA GB300"
    path = str(tmp_path / "tuned.json")
    assert autotune.lookup(key, path) is None
    entry = {"smoother_degree": 5, "cheb_ratio": 8.0, "ms": 170.0, "n_samples": 256,
             "schedule": {"uni_run": 8, "uni_waves": 4, "vec_rows": 128, "vcycle_rows": 16}}
    autotune.save(key, entry, path)
    other = autotune.cache_key(WORKLOADS["torus_p3_512x256_s1024"], 1024, "NVIDIA GB300")
    autotune.save(other, dict(entry, smoother_degree=6), path)
    assert autotune.lookup(key, path) == entry
    assert autotune.lookup(other, path)["smoother_degree"] == 6
    assert set(json.load(open(path))) == {key, other}


def test_committed_cache_entries_are_well_formed():
    from paper_2605_24882_gb300 import autotune
    if not os.path.exists(autotune.CACHE):
        return
    for key, e in json.load(open(autotune.CACHE)).items():
        kind, p, elems, levels, samples, precision, gpu = key.split("/")
        assert kind in ("sphere", "torus") and p[0] == "p" and levels[0] == "L" and samples[0] == "s"
        assert 1 <= e["smoother_degree"] <= 8 and e["cheb_ratio"] > 1
        sc = e["schedule"]
        assert 1 <= sc["uni_run"] <= 8 and 1 <= sc["uni_waves"] <= 64
        assert 32 <= sc["vec_rows"] <= 4096 and 8 <= sc["vcycle_rows"] <= 1024
        assert sc.get("tail_fused", 1) in (0, 1)


def test_schedule_knobs_are_abi_fields():
    # every knob the autotuner sweeps (and a cache entry may set) is a field of
    # the ABI's wm_schedule, so set_schedule cannot silently drop one
    from paper_2605_24882_gb300 import _capi, autotune
    fields = [n for n, _ in _capi.Schedule._fields_]
    assert set(autotune.SCHEDULE_CHOICES) == set(fields)
    if os.path.exists(autotune.CACHE):
        for e in json.load(open(autotune.CACHE)).values():
            assert set(e["schedule"]) <= set(fields)
