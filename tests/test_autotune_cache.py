"""The autotuner's cache of choices (host logic; no GPU): keys by GPU name
and problem shape class, and the JSON file's round trip."""
import json
import types

import numpy as np

from paper_1511_03296_gb300 import fbs


def _grid(vertex_counts):
    return types.SimpleNamespace(n_images=len(vertex_counts), vertex_counts=list(vertex_counts))


def _t(*channels):
    return [np.zeros((c, 2, 2), np.float32) for c in channels]


def test_key_classes():
    k = fbs.tuning_key(_grid([105966]), _t(3), device_name="GB300")
    assert k == "GB300|images~2^0|vertices~2^17|row=4"
    # shape classes: image count and vertices in powers of two, padded row
    assert fbs.tuning_key(_grid([70000, 50000]), _t(1, 2), "GB300") == \
        "GB300|images~2^1|vertices~2^17|row=2"
    assert fbs.tuning_key(_grid([1000] * 64), _t(*([1] * 63 + [21])), "GB300") == \
        "GB300|images~2^6|vertices~2^16|row=24"
    # another GPU or another size class is another key
    assert fbs.tuning_key(_grid([105966]), _t(3), "B200") != k
    assert fbs.tuning_key(_grid([4 * 105966]), _t(3), "GB300") != k


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    assert fbs._cache_read(path) == {}
    a = {"pcg_launch": 2, "pcg_form": 0, "phase_blocks": 2, "solve_ms": 0.5, "candidates": 6}
    b = {"pcg_launch": 1, "pcg_form": 1, "phase_blocks": 1, "solve_ms": 2.0, "candidates": 6}
    fbs._cache_write(path, "k1", a)
    fbs._cache_write(path, "k2", b)
    got = fbs._cache_read(path)
    assert got["k1"] == {k: a[k] for k in ("pcg_launch", "pcg_form", "phase_blocks", "solve_ms")}
    assert got["k2"]["pcg_form"] == 1
    assert json.load(open(path))["format"] == "fbs autotune cache 1"
    # a damaged file reads as empty, and is rewritten on the next store
    open(path, "w").write("{not json")
    assert fbs._cache_read(path) == {}
    fbs._cache_write(path, "k3", a)
    assert list(fbs._cache_read(path)) == ["k3"]
