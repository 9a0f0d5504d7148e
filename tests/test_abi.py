"""The C ABI: the library loads and exports every declared entry point, and
the host-only calls behave as documented (no GPU needed)."""
import ctypes
import os
import re

import pytest

import paper_2001_10635_b300 as R
from paper_2001_10635_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"REACH_API\s+[\w\s\*]*?\b(reach_\w+)\s*\(", text))
    return names


def test_library_builds_and_loads():
    B.build()
    assert os.path.exists(R.LIB_PATH)
    R.lib()


def test_every_declared_symbol_is_exported():
    names = declared_symbols()
    assert {"reach_mm", "reach_cgb", "reach_mc", "reach_system_create"} <= names
    L = ctypes.CDLL(R.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def test_mc_sample_bound():
    assert R.reach_mc_samples(1, 0.1, 0.1) == 60
    assert R.reach_mc_samples(16, 0.05, 0.01) == 5166
    assert R.reach_mc_samples(0, 0.1, 0.1) == -1
    assert R.reach_mc_samples(4, 1.5, 0.1) == -1


def test_options_are_validated():
    old = R.reach_get_option(R.OPT_STEPS_PER_LAUNCH)
    R.reach_set_option(R.OPT_STEPS_PER_LAUNCH, 3)
    assert R.reach_get_option(R.OPT_STEPS_PER_LAUNCH) == 3
    R.reach_set_option(R.OPT_STEPS_PER_LAUNCH, old)
    bad = [(R.OPT_STEPS_PER_LAUNCH, -1), (R.OPT_KERNEL, 5), (R.OPT_BLOCK, 33), (R.OPT_TILE, 4), (R.OPT_MC_SB, 4),
           (R.OPT_MC_LAYOUT, 11), (R.OPT_SERVE_QUEUE_BLOCKS, -1), (R.OPT_SERVE_QUEUE_N, 4097),
           (R.OPT_SERVE_MAX_WIDE, -1), (R.OPT_BATCH_CLUSTER_FROM, -1), (R.OPT_ONE_LAUNCH, 3),
           (R.OPT_SERVE_PRIORITY, 4), (R.OPT_SERVE_WIDE_EXCLUSIVE, 2), (99, 1)]
    for key, val in bad:
        with pytest.raises(R.ReachError):
            R.reach_set_option(key, val)


def test_option_defaults():
    # the defaults the header documents
    assert R.reach_get_option(R.OPT_SERVE_QUEUE_BLOCKS) == 64
    assert R.reach_get_option(R.OPT_SERVE_QUEUE_N) == 512
    assert R.reach_get_option(R.OPT_MC_LAYOUT) == 0 and R.reach_get_option(R.OPT_ONE_LAUNCH) == 0
    assert R.reach_get_option(R.OPT_SERVE_WIDE_EXCLUSIVE) == 1 and R.reach_get_option(R.OPT_SERVE_LIGHT) == 1 << 15
    assert R.reach_get_option(R.OPT_SERVE_MAX_WIDE) == 0


def test_strerror_names_every_code():
    for code in range(0, -8, -1):
        assert R.strerror(code) != "unknown status"
