"""Host logic of bench.py's recorded ncu counters: a kernel's DRAM traffic
and instruction count are reported only while the digest of its sources
equals the one recorded with the counters, and the instruction-issue
roofline is the recorded count x units / time against 4 warp instructions
per SM per clock."""
import json
import os
import types

import pytest

import bench
from paper_1612_03399_gb300 import build as B


def recorded():
    with open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")) as f:
        return json.load(f)


def test_counters_follow_the_source_digest(monkeypatch):
    d = recorded()
    key = "force"
    assert key in d["kernels"] and key in d["instructions"]
    # sources as recorded: the counters are reported
    monkeypatch.setattr(B, "kernel_digest", lambda k: d["digests"][k])
    assert bench.ncu_traffic(key) == d["kernels"][key]
    assert bench.ncu_instructions(key) == d["instructions"][key]
    # any change to the kernel's sources: nothing is reported
    monkeypatch.setattr(B, "kernel_digest", lambda k: "0" * 64)
    assert bench.ncu_traffic(key) is None
    assert bench.ncu_instructions(key) is None


def test_every_recorded_kernel_has_a_digest_and_sources():
    d = recorded()
    for key in d["kernels"]:
        assert key in d["digests"], key
        assert key in B.KERNEL_SOURCES, key
    for key in d["instructions"]:
        assert key in d["kernels"], key


def test_issue_roofline_arithmetic(monkeypatch):
    d = recorded()
    monkeypatch.setattr(B, "kernel_digest", lambda k: d["digests"][k])
    props = types.SimpleNamespace(multi_processor_count=152)
    monkeypatch.setattr(bench.torch.cuda, "get_device_properties", lambda i: props)
    ipu = d["instructions"]["marker"]
    r = bench.issue_roofline("marker", 1_280_000, 0.5, {"sm_mhz": 2000.0}, 0)
    peak = 152 * 4 * 2000e6
    assert r["peak"] == pytest.approx(peak)
    assert r["achieved"] == pytest.approx(ipu * 1_280_000 / 0.5e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / peak)
    # no clock sample and no maximum clock: no roofline
    assert bench.issue_roofline("marker", 1, 0.5, {}, 0) is None
