"""Host-side rules of bench.py that shape what it measures, on CPU: the
per-graph grid caps of the batched workload and the fused kernel's traffic
figure, which is reported only while the profile matches the source."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_batch_caps_cover_the_batch_and_stay_valid():
    """The caps grow with n, are multiples of 16, lie between the default
    minimum of 50 boxes and the library's 640, and give every graph at least
    1.5 times the box counts the batch recipe's graphs were seen to reach
    (120 boxes below n = 500, 135 up to 2000, 150 up to 5000, 180 up to
    20,000)."""
    ns = np.unique(np.round(np.exp(np.linspace(np.log(200), np.log(20_000), 200))).astype(int))
    caps = bench.batch_caps(ns)
    assert caps.dtype == np.int32 and caps.shape == ns.shape
    assert np.all(np.diff(caps) >= 0)
    assert np.all(caps % 16 == 0)
    assert caps.min() >= 50 and caps.max() <= 640
    seen = np.where(ns < 500, 120, np.where(ns < 2000, 135, np.where(ns < 5000, 150, 180)))
    assert np.all(caps >= 1.5 * seen - 16), (ns[caps < 1.5 * seen - 16], caps[caps < 1.5 * seen - 16])


def test_fused_traffic_reported_only_for_the_profiled_source(tmp_path, monkeypatch):
    """The committed profile's traffic figure is read while its source hash
    equals the current kernel source's; a profile of another source gives
    no figure."""
    text = open(bench.FUSED_PROFILE).read()
    assert bench.ncu_traffic_per_launch() is not None
    stale = tmp_path / "profile.md"
    stale.write_text(text.replace(f"kernel_source_hash = {bench.kernel_hash()}", "kernel_source_hash = 0000000000000000"))
    monkeypatch.setattr(bench, "FUSED_PROFILE", str(stale))
    assert bench.ncu_traffic_per_launch() is None
