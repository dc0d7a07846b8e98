"""Host-side pieces of bench.py that run without a GPU: the traffic figure is
only reported for the source it was measured on, every file it hashes
exists, MAPE follows its stated definition, and the oracle's thread count
is a usable positive number."""

import json
import os

import numpy as np

import bench


def test_traffic_is_reported_only_for_the_measured_source():
    p = os.path.join(bench.ROOT, "profiles", "traffic.json")
    d = json.load(open(p))
    k, rec = next(iter(d.items()))
    assert bench.traffic_for(k, rec["src_sha"]) == rec["dram_bytes_per_launch"]
    assert bench.traffic_for(k, "0" * 16) is None
    assert bench.traffic_for("no_such_kernel", rec["src_sha"]) is None


def test_hashed_sources_exist():
    for f in bench.REC_SRC + bench.EYE_SRC:
        assert os.path.exists(os.path.join(bench.ROOT, f)), f
    assert len(bench.src_sha(bench.REC_SRC)) == 16


def test_mape_definition():
    ref = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0]])
    eps = 1e-2 * ref.mean()
    x = ref * 1.1
    np.testing.assert_allclose(bench.mape(x, ref), np.mean(0.1 * ref / (ref + eps)))
    assert bench.mape(ref, ref) == 0.0


def test_oracle_thread_count():
    n = bench.oracle_threads()
    assert 1 <= n <= 64
