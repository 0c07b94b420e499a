import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built libmb4")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on one CPU core")
    config.addinivalue_line("markers", "oracle_long(job): compares with a long oracle trajectory that "
                                       "tests/oracle_jobs.py computes in a spawned process")


def pytest_collection_finish(session):
    """Start the long oracle trajectories that the selected tests need, in spawned
    processes, before the first test runs: they then overlap the other GPU tests."""
    if session.config.option.collectonly:
        return
    jobs = set()
    for item in session.items:
        for m in item.iter_markers("oracle_long"):
            jobs.update(m.args)
    if jobs:
        import oracle_jobs
        oracle_jobs.start(tuple(sorted(jobs)))


def pytest_sessionfinish(session, exitstatus):
    mod = sys.modules.get("oracle_jobs")
    if mod is not None:
        mod.shutdown()
