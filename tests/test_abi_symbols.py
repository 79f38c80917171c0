"""The C-ABI library loads and exports every function include/rafi.h declares.

No compute call is made: this runs on a machine without a GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(rf_\w+)\s*\(", text, flags=re.M))
    return names


@pytest.fixture(scope="module")
def built_lib():
    from paper_2605_30294_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("rf_create", "rf_destroy", "rf_resize", "rf_get_device_queues", "rf_exchange",
                 "rf_num_active", "rf_segment", "rf_stats", "rf_push", "rf_snapshot", "rf_restore",
                 "rf_last_error", "rf_c1_run", "rf_c0_render"):
        assert must in names


def test_library_exports_every_declared_symbol(built_lib):
    missing = [n for n in sorted(_declared()) if not hasattr(built_lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(built_lib):
    from paper_2605_30294_gb300 import rafi

    declared = _declared()
    assert declared <= set(rafi._SIGS), declared - set(rafi._SIGS)
    for n in declared:
        assert hasattr(rafi, n), n


def test_host_only_calls_without_gpu(built_lib):
    # argument validation and the host-side Zipf table need no device
    from paper_2605_30294_gb300 import rafi

    import oracle

    thr = rafi.rf_c1_zipf_thresholds(64, 1.1)
    assert thr == [int(x) for x in oracle.zipf_thresholds(64, 1.1)]
    with pytest.raises(rafi.RafiError) as e:
        rafi.rf_create(0, 64, 10)
    assert e.value.status == rafi.RF_ERR_ARG
    with pytest.raises(rafi.RafiError) as e:
        rafi.rf_create(4, 40, 10)
    assert e.value.status == rafi.RF_ERR_ARG
    assert "multiple of 16" in rafi.rf_last_error()
    assert rafi.rf_launch_count() == 0
