"""The committed ncu traffic records still describe the kernels as built.

bench.py reports a copy kernel's DRAM traffic only while the text the kernel
is compiled from hashes to the value recorded beside the capture; a change to
those sources must come with a new capture. This checks that every record
matches, so the roofline line does not silently lose its traffic figure."""
import glob
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_records_match_their_sources():
    paths = sorted(glob.glob(os.path.join(ROOT, "profiles", "*_traffic.json")))
    assert paths
    for p in paths:
        d = json.load(open(p))
        assert bench.kernel_source_sha(d["sources"]) == d["source_sha256"], os.path.basename(p)
        assert 0.5 < d["traffic_over_algorithmic"] < 1.5
        cited = [w for w in d["from"].split() if w.startswith("profiles/")]
        assert cited and all(os.path.exists(os.path.join(ROOT, w)) for w in cited), d["from"]
        assert bench.copy_traffic(d["kernel"], 1.0) == d["traffic_over_algorithmic"]
