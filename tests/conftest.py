import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_addoption(parser):
    parser.addoption("--runslow", action="store_true", default=False,
                     help="also run tests marked slow (or set MPR_RUN_SLOW=1)")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running or memory-heavy; skipped unless "
                                       "--runslow or MPR_RUN_SLOW=1")


def pytest_collection_modifyitems(config, items):
    if config.getoption("--runslow") or os.environ.get("MPR_RUN_SLOW") == "1":
        return
    skip = pytest.mark.skip(reason="slow: run with --runslow or MPR_RUN_SLOW=1")
    for item in items:
        if "slow" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle


# Near-threshold sites that single-sweep parity tests excuse, per test: printed at the end of the
# session, so a rise in their number is visible even while it stays under a test's bound.
_EXCUSED = []


@pytest.fixture
def excusal_log(request):
    def log(what, excused, total, bound):
        _EXCUSED.append((request.node.nodeid, what, int(excused), int(total), float(bound)))
    return log


# Accuracy gaps of the statistical parity tests (setup, metric, relative gap, bound), printed last.
_GAPS = []


@pytest.fixture
def gap_log(request):
    def log(what, metric, gap, bound):
        _GAPS.append((request.node.nodeid, what, metric, float(gap), float(bound)))
    return log


def pytest_terminal_summary(terminalreporter):
    _excusal_summary(terminalreporter)
    if _GAPS:
        path = os.environ.get("MPR_GAPS_JSON")
        if path:
            import json

            with open(path, "w") as fh:
                json.dump(_GAPS, fh, indent=0)
        tr = terminalreporter
        tr.section("statistical parity: relative gaps (bound)")
        for nodeid, what, metric, gap, bound in _GAPS:
            tr.write_line(f"{what:34s} {metric:8s} {gap:+.2e} ({bound:g})")


def _excusal_summary(terminalreporter):
    if not _EXCUSED:
        return
    path = os.environ.get("MPR_EXCUSAL_JSON")
    if path:
        import json

        with open(path, "w") as fh:
            json.dump(_EXCUSED, fh, indent=0)
    tr = terminalreporter
    tr.section("excused near-threshold sites (single-sweep parity)")
    for nodeid, what, n, total, bound in _EXCUSED:
        tr.write_line(f"{n:7d} of {total:10d} ({n / max(total, 1):.2e}; bound {bound:g}) "
                      f"{what:10s} {nodeid}")
