"""Host-side pieces of bench.py that decide what the JSON line claims: the kernel-version hash
that ties stored ncu counters to the code they came from, and the lookup of those counters."""
import json
import os

import pytest

import bench


def test_kernel_id_is_a_stable_hash_of_the_kernel_sources():
    a = bench.sweep_kernel_id()
    assert a == bench.sweep_kernel_id() and len(a) == 16
    assert a != bench.sweep_kernel_id("mpr::sweep_f32_tma_kernel")


def test_stored_counters_belong_to_their_kernel_version():
    # counters are reported only for the kernel version they were captured from; a stale record
    # (sources changed since) makes bench.py report traffic null, which this test allows
    with open(os.path.join(bench.ROOT, "profiles", "dram_traffic.json")) as fh:
        d = json.load(fh)
    e = d["L4096_p0.9_HDS"]
    assert e["kernel"] == "mpr::sweep_f32_kernel"
    assert bench.stored_counters("0" * 16, "mpr::sweep_f32_kernel", "L4096_p0.9_HDS") == {}
    assert bench.stored_counters(e["kernel_id"], "mpr::sweep_kernel", "L4096_p0.9_HDS") == {}
    if e["kernel_id"] != bench.sweep_kernel_id():
        pytest.skip("stored counters are from another kernel version (bench reports null)")
    got = bench.stored_counters(bench.sweep_kernel_id(), "mpr::sweep_f32_kernel", "L4096_p0.9_HDS")
    assert got and got["bytes_per_launch"] == e["bytes_per_launch"]
    assert 0.0 < got["issue_active"] <= 1.0
    # algorithmic bytes of one 4096^2 FP16 pass: (N/2)(2(2 + p) + 1/8) = 49.7 MB; the measured
    # DRAM bytes are below it (the 33.5 MB state stays in the 129 MB L2 between passes, and the
    # capture keeps the cache as the previous pass left it) and never far above it (no re-reads)
    alg = 4096 * 4096 / 2 * (2 * 2.9 + 1 / 8)
    assert 0.1 * alg < got["bytes_per_launch"] < 1.5 * alg
