"""Host-side pieces of bench.py that need no GPU: the algorithmic flop count behind the
roofline, and the DRAM-traffic lookup that is valid only for the kernel sources it was taken on."""
import json
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_algorithmic_flops_are_two_ffts_of_5_n_log2_n():
    import bench
    for F in (64, 128, 256, 512):
        N = F * F
        assert bench.algorithmic_flops_per_eval(F) == pytest.approx(2 * 5 * N * math.log2(N))
    assert bench.algorithmic_flops_per_eval(256) == pytest.approx(10.49e6, rel=1e-3)


def test_traffic_is_reported_only_for_the_kernel_sources_and_launch_size_it_was_measured_on(monkeypatch):
    import bench
    d = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    monkeypatch.setattr(bench, "kernel_hash", lambda: d["kernel_sha"])
    ev = d["config2:col_adj"]["evaluations_per_launch"]
    v = bench.ncu_traffic("col_adj", "config2", ev)
    assert v == d["config2:col_adj"]["dram_bytes_per_launch"] and v > 0
    assert bench.ncu_traffic("col_adj", "config2", 0.97 * ev) == v          # a ragged last batch
    assert bench.ncu_traffic("col_adj", "config2", 0.8 * ev) is None         # other launch sizes
    monkeypatch.setattr(bench, "kernel_hash", lambda: "0" * 16)
    assert bench.ncu_traffic("col_adj", "config2", ev) is None
    monkeypatch.undo()
    assert bench.ncu_traffic("no_such_kernel", "config2", ev) is None


def test_camera_frames_are_seeded_and_hit_both_thresholds():
    from synthetic import workloads as syn
    a = syn.camera_frames(3, 64, seed=4)
    b = syn.camera_frames(3, 64, seed=4)
    assert a.dtype == np.float32 and a.shape == (3, 64, 64)
    assert np.array_equal(a, b)
    assert (a >= 65535).any() and (a < 4).any() and a.max() == 65535
