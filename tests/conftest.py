import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (runs on the B300 box)")
    config.addinivalue_line("markers", "slow: long-running CPU case")


def pytest_sessionstart(session):
    # the tests load the in-tree libreach.so: build it when it is missing or
    # older than its sources (a no-op otherwise); the package itself never
    # falls back when it is absent.  Parallel workers leave it to the main
    # process, which starts first.
    if hasattr(session.config, "workerinput"):
        return
    from paper_2001_10635_b300 import build as B
    B.build()
