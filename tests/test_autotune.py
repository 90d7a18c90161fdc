"""The batched autotuner's host logic: cache keys, the coordinate search and
the JSON cache (no GPU: the timing function is a stand-in)."""
import os

from paper_2206_00975_gb300 import autotune


def test_key_buckets_shapes_by_padded_length_and_panel():
    k1 = autotune.key_for([(2048, 9), (65533, 129)], "f64", "sm_103")
    assert k1 == "sm_103|mp=65536|npanel=256|f64"
    k2 = autotune.key_for([(40000, 100), (50000, 120)], "f64", "sm_103")
    assert k2 == "sm_103|mp=65536|npanel=128|f64"
    assert autotune.key_for([(40000, 100)], "f32", "sm_103") != autotune.key_for([(40000, 100)], "f64", "sm_103")


def test_coordinate_search_finds_the_best_setting_of_each_knob():
    # a separable cost with its minimum at panel 2, sketch 4, dense 1
    cost = {"panel": {1: 3.0, 2: 1.0, 4: 2.0}, "sketch_ctas_per_sm": {0: 2.0, 4: 0.5, 2: 1.0},
            "dense_ctas_per_sm": {0: 1.0, 2: 0.7, 1: 0.2}}
    calls = []

    def measure(s):
        calls.append(dict(s))
        return sum(cost[k][v] for k, v in s.items())
    best, t, tried = autotune.coordinate_search(measure)
    assert best == {"panel": 2, "sketch_ctas_per_sm": 4, "dense_ctas_per_sm": 1}
    assert abs(t - 1.7) < 1e-12
    assert len(calls) == len(tried) == 1 + 2 + 2 + 2   # start, then the other values of each knob


def test_cache_round_trip(tmp_path):
    path = os.path.join(str(tmp_path), "sub", "tuning.json")
    assert autotune.load_cache(path) == {}
    autotune.save_cache({"k": {"setting": {"panel": 2}}}, path)
    assert autotune.load_cache(path)["k"]["setting"] == {"panel": 2}
