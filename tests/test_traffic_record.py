"""The committed per-tier DRAM traffic record of the backward
(profiles/backward_traffic.json) belongs to the kernel source in the tree:
bench.py reports roofline.traffic only while the record's source hash
matches, so a kernel change without a new capture would silently drop it."""
import json
import os

import bench
from paper_2401_05345_gb300 import autotune

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _record():
    with open(os.path.join(ROOT, "profiles", "backward_traffic.json")) as f:
        return json.load(f)


def test_traffic_record_matches_the_kernel_source():
    d = _record()
    h = bench.kernel_source_hash()
    assert d["kernel_hash"] == h, "kernel sources changed since the traffic capture: recapture it"
    tiers = {k: v for k, v in d.items() if isinstance(v, dict)}
    assert tiers and all(v["kernel_hash"] == h for v in tiers.values())


def test_traffic_record_covers_every_autotune_candidate():
    d = _record()
    names = {autotune.opts_name(o) for o in autotune.default_candidates()}
    missing = {n for n in names if n not in d and not n.startswith("cluster")}
    assert not missing, sorted(missing)
    for n in names & set(d):
        e = d[n]
        assert e["dram_bytes_per_launch"] == e["dram_read"] + e["dram_write"] > 0
