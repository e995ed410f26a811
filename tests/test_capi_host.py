"""Host-side checks of the C ABI: the library builds, loads, exports every
symbol that include/de.h declares, and rejects invalid configurations before
touching a GPU.  CPU only."""
import os
import re

import numpy as np
import pytest

from paper_2405_16551_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^DE_API\s+[\w\s\*]+?\b(de_\w+)\s*\(", txt, flags=re.M)
    return names


def test_library_exports_every_declared_symbol():
    lib = capi.load()
    declared = _header_functions()
    assert len(declared) >= 18
    for name in declared:
        assert hasattr(lib, name), name
    assert set(capi.exported_symbols()) <= set(declared)


def test_version_and_status_strings():
    assert capi.de_version().startswith("de_gb300")
    lib = capi.load()
    assert lib.de_status_string(capi.DE_ERR_INVALID_ARG) == b"DE_ERR_INVALID_ARG"
    assert lib.de_status_string(capi.DE_OK) == b"DE_OK"


@pytest.mark.parametrize(
    "kw,msg",
    [
        (dict(np_=3, d=10), "np"),
        (dict(np_=64, d=0), "d must"),
        (dict(np_=64, d=5000), "d must"),
        (dict(np_=64, d=10, f=-0.1), "F must"),
        (dict(np_=64, d=10, f=2.5), "F must"),
        (dict(np_=64, d=10, cr=1.5), "CR must"),
        (dict(np_=64, d=10, lo=1.0, hi=1.0), "bounds"),
        (dict(np_=64, d=10, lo=float("nan")), "bounds"),
        (dict(np_=64, d=10, objective=9), "objective"),
        (dict(np_=64, d=10, scale=0.0), "scale"),
        (dict(np_=64, d=10, run_id=1 << 20), "run_id"),
        (dict(np_=64, d=10, precision=7), "precision"),
        (dict(np_=64, d=10, max_generations=-1), "max_"),
        (dict(np_=64, d=2, shift=np.array([0.0, np.inf])), "shift"),
        (dict(np_=64, d=2, rot=np.array([[1.0, 0.0], [np.nan, 1.0]])), "rotation"),
    ],
)
def test_invalid_config_rejected_on_host(kw, msg):
    cfg = capi.make_config(**kw)
    with pytest.raises(capi.DEError) as ei:
        capi.de_init(cfg)
    assert ei.value.status == capi.DE_ERR_INVALID_ARG
    assert msg in str(ei.value)


def test_null_arguments_rejected():
    lib = capi.load()
    assert lib.de_init(None, None, None) == capi.DE_ERR_INVALID_ARG
    assert lib.de_step(None, 1) == capi.DE_ERR_INVALID_ARG
    assert lib.de_destroy(None) == capi.DE_OK
    assert b"NULL" in lib.de_last_error(None)
