"""Host logic of the autotuner (paper_1711_00121_gb300.tune): the coordinate
search, the cache key and file, and the timing updates.  No GPU needed."""
import json

import numpy as np

from paper_1711_00121_gb300 import tune
from synth import chung_lu_digraph


def test_coordinate_search_finds_the_minimum_of_a_separable_cost():
    space = {"defer": [16, 8, 24, 32], "tc": [2, 1], "prep_item": [1024, 512, 2048]}
    cost = {"defer": {8: 3.0, 16: 2.0, 24: 1.0, 32: 1.5}, "tc": {1: 0.5, 2: 0.0},
            "prep_item": {512: 0.2, 1024: 0.1, 2048: 0.0}}
    calls = []

    def measure(k):
        calls.append(dict(k))
        return sum(cost[n][v] for n, v in k.items())

    best, t, seen = tune.coordinate_search(space, measure)
    assert best == {"defer": 24, "tc": 2, "prep_item": 2048}
    assert abs(t - 1.0) < 1e-12
    # each distinct candidate is timed once: start + 3 + 1 + 2
    assert len(calls) == len(seen) == 7


def test_coordinate_search_keeps_the_start_when_nothing_is_faster():
    space = {"a": [1, 2, 3], "b": [0, 1]}
    best, t, _ = tune.coordinate_search(space, lambda k: k["a"] + k["b"], start={"a": 1, "b": 0})
    assert best == {"a": 1, "b": 0} and t == 1


def test_key_buckets_n_by_powers_of_two():
    assert tune.n_bucket(20000) == 32768 and tune.n_bucket(32768) == 32768
    assert tune.n_bucket(5) == 128
    assert tune.key("stream", "GB300", 20000, 20, 32, 1) == "stream|GB300|n32768|K20|s32|v1"


def test_cache_round_trip_and_lookup(tmp_path):
    path = str(tmp_path / "tuned.json")
    assert tune.lookup("stream", "GB300", 1000, 15, 32, 1, path) is None
    entries = {tune.key("stream", "GB300", 1000, 15, 32, 1): {"knobs": {"defer": 8, "tc": 1},
                                                            "us_per_update": 1.0}}
    tune.save(entries, path)
    with open(path) as f:
        assert json.load(f) == entries
    assert tune.lookup("stream", "GB300", 900, 15, 32, 1, path) == {"defer": 8, "tc": 1}
    assert tune.lookup("stream", "GB300", 1000, 16, 32, 1, path) is None


def test_timing_updates_insert_absent_edges_then_delete_them():
    n = 800
    s, d = chung_lu_digraph(n, 6000, 2.1, 2.1, 5)
    ups = tune.timing_updates(n, s, d, 40, seed=3)
    assert ups.shape == (40, 3)
    have = set(zip(s.tolist(), d.tolist()))
    ins, dels = ups[:20], ups[20:]
    assert np.all(ins[:, 2] == 1) and np.all(dels[:, 2] == -1)
    assert np.array_equal(ins[:, :2], dels[:, :2])
    pairs = [tuple(x) for x in ins[:, :2].tolist()]
    assert len(set(pairs)) == 20 and all(p not in have and p[0] != p[1] for p in pairs)


def test_stream_space_respects_the_pending_limit():
    sp = tune.stream_space(K=200, num_sms=152)
    assert all(g * 201 <= 4096 for g in sp["defer"]) and sp["prep_ctas"] == [0, 152]
