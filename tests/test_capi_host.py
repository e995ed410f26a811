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
        (dict(np_=64, d=10, objective=99), "objective"),
        (dict(np_=64, d=10, scale=0.0), "scale"),
        (dict(np_=64, d=10, run_id=1 << 20), "run_id"),
        (dict(np_=64, d=10, precision=7), "precision"),
        (dict(np_=64, d=10, max_generations=-1), "max_"),
        (dict(np_=64, d=2, shift=np.array([0.0, np.inf])), "shift"),
        (dict(np_=64, d=2, rot=np.array([[1.0, 0.0], [np.nan, 1.0]])), "rotation"),
        (dict(np_=64, d=10, objective=4), "d = 20"),
        (dict(np_=64, d=20, objective=4, precision=2), "FP64 only"),
        (dict(np_=64, d=20, objective=4, rot=np.eye(20)), "no rotation"),
        (dict(np_=64, d=10, strategy=3), "strategy"),
        (dict(np_=64, d=10, objective=21), "objective"),
        (dict(np_=64, d=10, objective=5, precision=1), "FP64 only"),
        (dict(np_=64, d=10, objective=18, precision=2), "FP64 only"),
        (dict(np_=64, d=6, objective=17), "too small"),
        (dict(np_=64, d=10, objective=18, scale=0.5), "scale 1"),
        (dict(np_=64, d=4, objective=1, perm=np.arange(4)), "hybrid functions only"),
        (dict(np_=64, d=10, objective=15, perm=np.array([0, 1, 1, 3, 4, 5, 6, 7, 8, 9])), "permutation"),
        (dict(np_=64, d=10, objective=15, perm=np.array([0, 1, 2, 3, 4, 5, 6, 7, 8, 10])), "permutation"),
        (dict(np_=64, d=2, objective=19, shift=np.array([0.0, 1.0, np.nan, 0, 0, 0, 0, 0])), "shift"),
        (dict(np_=64, d=10, strategy=-1), "strategy"),
    ],
)
def test_invalid_config_rejected_on_host(kw, msg):
    cfg = capi.make_config(**kw)
    with pytest.raises(capi.DEError) as ei:
        capi.de_init(cfg)
    assert ei.value.status == capi.DE_ERR_INVALID_ARG
    assert msg in str(ei.value)


@pytest.mark.parametrize(
    "kw",
    [
        dict(jde=True, surrogate_k=4),
        dict(strategy=capi.DE_BEST1BIN, surrogate_k=8),
    ],
)
def test_variants_with_a_surrogate_are_unsupported_on_host(kw):
    cfg = capi.make_config(64, 20, **kw)
    with pytest.raises(capi.DEError) as ei:
        capi.de_init(cfg)
    assert ei.value.status == capi.DE_ERR_UNSUPPORTED
    assert "surrogate" in str(ei.value)


def test_null_arguments_rejected():
    lib = capi.load()
    assert lib.de_init(None, None, None) == capi.DE_ERR_INVALID_ARG
    assert lib.de_step(None, 1) == capi.DE_ERR_INVALID_ARG
    assert lib.de_destroy(None) == capi.DE_OK
    assert b"NULL" in lib.de_last_error(None)


@pytest.mark.parametrize(
    "args,status,msg",
    [
        ((7, 1, 10, 1.0), "DE_ERR_INVALID_ARG", "precision"),
        ((0, 1, 10, 1.0), "DE_ERR_UNSUPPORTED", "FP64"),
        ((1, 4, 10, 1.0), "DE_ERR_INVALID_ARG", "objective"),
        ((1, 1, 0, 1.0), "DE_ERR_INVALID_ARG", "d must"),
        ((2, 1, 4097, 1.0), "DE_ERR_INVALID_ARG", "d must"),
        ((1, 2, 300, 1.0), "DE_ERR_UNSUPPORTED", "Rosenbrock"),
        ((1, 1, 10, 0.0), "DE_ERR_INVALID_ARG", "scale"),
        ((1, 1, 10, float("inf")), "DE_ERR_INVALID_ARG", "scale"),
    ],
)
def test_eval_noalloc_rejects_arguments_on_host(args, status, msg):
    """de_eval_noalloc checks its scalar arguments before any CUDA call."""
    lib = capi.load()
    prec, obj, d, scale = args
    st = lib.de_eval_noalloc(prec, obj, d, scale, None, None, None, d, 4, None, None)
    assert lib.de_status_string(st).decode() == status
    assert msg in lib.de_last_error(None).decode()


def test_eval_noalloc_empty_and_negative_n_on_host():
    lib = capi.load()
    assert lib.de_eval_noalloc(1, 1, 10, 1.0, None, None, None, 10, 0, None, None) == capi.DE_OK
    assert lib.de_eval_noalloc(1, 1, 10, 1.0, None, None, None, 10, -1, None, None) == capi.DE_ERR_INVALID_ARG


@pytest.mark.parametrize(
    "args,status",
    [
        ((1, 5, 1), "DE_ERR_INVALID_ARG"),      # one island
        ((4, 0, 1), "DE_ERR_INVALID_ARG"),      # no interval
        ((4, 5, 0), "DE_ERR_INVALID_ARG"),      # no migrants
        ((4, 5, 33), "DE_ERR_INVALID_ARG"),     # above 32
        ((4, 5, 40), "DE_ERR_INVALID_ARG"),     # above np / 2
    ],
)
def test_island_arguments_rejected_on_host(args, status):
    cfg = capi.make_config(64, 10)
    with pytest.raises(capi.DEError) as ei:
        capi.de_init_islands(cfg, *args)
    assert status in str(ei.value)


def test_islands_outside_the_fp64_path_are_unsupported_on_host():
    for kw in (dict(precision=capi.DE_PREC_BF16X3), dict(surrogate_k=4)):
        cfg = capi.make_config(64, 20, **kw)
        with pytest.raises(capi.DEError) as ei:
            capi.de_init_islands(cfg, 4, 5, 1)
        assert ei.value.status == capi.DE_ERR_UNSUPPORTED
    cfg = capi.make_config(64, 20, run_id=(1 << 20) - 2)
    with pytest.raises(capi.DEError) as ei:
        capi.de_init_islands(cfg, 4, 5, 1)
    assert ei.value.status == capi.DE_ERR_INVALID_ARG


@pytest.mark.parametrize("migration", [-1, 2, 7])
def test_unknown_migration_strategy_rejected_on_host(migration):
    cfg = capi.make_config(64, 10)
    with pytest.raises(capi.DEError) as ei:
        capi.de_init_islands_ex(cfg, 4, 5, 1, migration)
    assert ei.value.status == capi.DE_ERR_INVALID_ARG and "migration" in str(ei.value)


def test_async_island_arguments_checked_like_sync_on_host():
    cfg = capi.make_config(64, 10)
    for args in ((1, 5, 1), (4, 0, 1), (4, 5, 33)):
        with pytest.raises(capi.DEError) as ei:
            capi.de_init_islands_ex(cfg, *args, capi.DE_MIGRATE_ASYNC)
        assert ei.value.status == capi.DE_ERR_INVALID_ARG
