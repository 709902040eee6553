"""The committed ncu summaries: every DRAM-traffic entry the benchmark may
report names an existing summary, a positive byte count per launch and the
source hash it was taken on (the benchmark reports the traffic only while
that hash matches the kernel's current source)."""
import json
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_traffic_entries_are_well_formed():
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    assert d
    for key, v in d.items():
        kernel, workload = key.split("@")
        assert kernel and workload
        assert v["bytes_per_launch"] > 0
        assert v["queries_per_launch"] > 0
        assert re.fullmatch(r"[0-9a-f]{16}", v["source_sha"]), key
        path = os.path.join(ROOT, v["profile"])
        assert os.path.isfile(path), path
        assert kernel in open(path).read().splitlines()[0]


def test_summaries_give_their_command():
    pdir = os.path.join(ROOT, "profiles")
    for f in os.listdir(pdir):
        if f.endswith(".md"):
            text = open(os.path.join(pdir, f)).read()
            assert "ncu " in text and "--clock-control none" in text, f
