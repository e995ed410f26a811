"""The largest problems the C ABI accepts (d = 4096, np = 2^20) and empty
inputs, against the CPU oracle: one generation with bit-exact indices, masks
and trials, fitness within the stated tolerance, selections outside the band."""
import numpy as np
import pytest

import oracle
from paper_2405_16551_gb300 import capi, problems

pytestmark = pytest.mark.gpu

REL64 = 1e-12
REL_SPLIT = {capi.DE_PREC_FP64: 1e-12, capi.DE_PREC_BF16X3: 1e-5, capi.DE_PREC_TF32X3: 1e-6}


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _one_generation(np_, d, obj, prec, rotate, seed, monkeypatch):
    monkeypatch.setenv("DE_GB300_PERSIST", "0")
    o = problems.shift(d, seed=seed)
    M = problems.rotation(d, seed=seed) if rotate else None
    X = problems.population(np_, d, seed=seed)
    fX, _ = oracle.evaluate(obj, X, o, M, threads=8)
    cfg = capi.make_config(np_, d, objective=obj, shift=o, rot=M, seed=seed, precision=prec, max_generations=10,
                           target_error=0.0, debug_capture=True, fp64_band=capi.DE_BAND_ALL)
    h = capi.de_init(cfg)
    try:
        capi.de_set_population(h, 0, X, fX)
        capi.de_set_generation(h, 0, 2)
        capi.de_step(h, 1)
        g = capi.de_get_debug(h)
        xn, fn = capi.de_get_population(h)
    finally:
        capi.de_destroy(h)
    r = oracle.step(X, fX, 0.5, 0.9, -100, 100, obj, o, M, seed=seed, generation=3, threads=8)
    assert np.array_equal(g["idx"], r["idx"]) and np.array_equal(g["jrand"], r["jrand"])
    assert np.array_equal(g["mask"], r["mask"]) and np.array_equal(g["trial"], r["trial"])
    fp64 = g["fp64_checked"].astype(bool)
    scale = np.abs(r["f_trial"]) + r["sabs_trial"]
    assert np.all(np.abs(g["f_trial"] - r["f_trial"]) <= np.where(fp64, REL64, REL_SPLIT[prec]) * scale)
    inband = np.abs(r["f_trial"] - fX) <= REL64 * scale
    assert np.array_equal(g["accept"][~inband], r["accept"][~inband])
    acc = g["accept"].astype(bool)
    assert np.array_equal(xn[acc], r["trial"][acc]) and np.array_equal(xn[~acc], X[~acc])


@pytest.mark.parametrize("prec", [capi.DE_PREC_FP64, capi.DE_PREC_BF16X3])
def test_largest_dimension(prec, monkeypatch):
    """d = 4096: one FP64 target per tile, sixteen N tiles of the split GEMM."""
    _need_gpu()
    _one_generation(12, 4096, 1, prec, True, 31, monkeypatch)


@pytest.mark.parametrize("prec,d", [(capi.DE_PREC_FP64, 2), (capi.DE_PREC_BF16X3, 16)])
def test_largest_population(prec, d, monkeypatch):
    """np = 2^20: the index map and the tile lists at their limit."""
    _need_gpu()
    _one_generation(1 << 20, d, 0, prec, prec != capi.DE_PREC_FP64, 32, monkeypatch)


@pytest.mark.parametrize("prec", [capi.DE_PREC_FP64, capi.DE_PREC_BF16X3])
def test_empty_evaluation_is_a_no_op(prec):
    torch = _need_gpu()
    h = capi.de_init(capi.make_config(16, 10, precision=prec, max_generations=1))
    try:
        fd = torch.full((4,), 7.0, dtype=torch.float64, device="cuda")
        xd = torch.zeros((4, 10), dtype=torch.float64, device="cuda")
        capi.de_eval(h, 0, xd.data_ptr(), 10, 0, fd.data_ptr())
        torch.cuda.synchronize()
        assert torch.all(fd == 7.0)
    finally:
        capi.de_destroy(h)


def test_fp64_rate_self_test():
    """The measured FP64 fused multiply-add rate is positive and of the order
    of the part's FP64 rate (GB300: about 1.25 TFLOP/s nominal)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    r = capi.de_selftest_fp64_rate()
    assert 0.2 < r < 5.0, r
