"""The MUFU throughput probe that bench.py runs for its roofline denominators.

It must run, report all four operations, and measure rates that are physically sensible: at most
the issue rate of 32 lanes per SM per clock at the maximum clock (a higher figure would mean the
compiler folded the chains away), and ex2 no slower than sin (on this part ex2 runs at twice the
sin rate)."""
import json
import os
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_mufu_probe_rates_are_sensible():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1910_08448_gb300 import _build

    r = subprocess.run([_build.PROBE], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    d = json.loads(r.stdout.strip().splitlines()[-1])
    sms = d["sms"]
    ceiling = sms * 32 * 2.2e9   # 32 lanes per SM at 2.2 GHz, above any clock of this part
    for op in ("sin", "cos", "ex2", "rcp"):
        rate = d[f"{op}_per_s"]
        assert 0.2 * sms * 16 * 1.0e9 < rate < ceiling, (op, rate)
    assert d["ex2_per_s"] >= 0.95 * d["sin_per_s"]
