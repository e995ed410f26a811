"""de_eval_noalloc: split-precision evaluation through the library's static
device scratch, with no handle and no allocation.

The entry point runs the same evaluation kernels as de_eval on a handle, so
its results must equal de_eval's bit for bit.  Each comparison makes two
calls in a row (different row counts and inputs, ragged last tiles), because
the second call reuses scratch that the first one wrote.  Through the C ABI
only.  This file is collected last; it must pass alone and after the others.
"""
import numpy as np
import pytest

import oracle
from paper_2405_16551_gb300 import capi, problems

pytestmark = pytest.mark.gpu

PRECS = [capi.DE_PREC_BF16X3, capi.DE_PREC_TF32X3]
REL_SPLIT = {capi.DE_PREC_BF16X3: 1e-5, capi.DE_PREC_TF32X3: 1e-6}
# largest n per call at d = 100 for the 16 MiB scratch (stated in de.h)
MAX_ROWS_D100 = {capi.DE_PREC_BF16X3: 36992, capi.DE_PREC_TF32X3: 18432}


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _padded(torch, X, ld):
    """Rows of X in device memory with row stride ld >= d (padding = NaN)."""
    n, d = X.shape
    buf = np.full((n, ld), np.nan)
    buf[:, :d] = X
    return torch.from_numpy(buf).cuda()


def _both(torch, h, prec, obj, d, scale, od, Md, X, ld):
    """f from de_eval (handle) and from de_eval_noalloc on the same rows."""
    n = len(X)
    xd = _padded(torch, X, ld)
    f_ref = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    f_na = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    capi.de_eval(h, 0, xd.data_ptr(), ld, n, f_ref.data_ptr())
    capi.de_eval_noalloc(prec, obj, d, scale, None if od is None else od.data_ptr(),
                         None if Md is None else Md.data_ptr(), xd.data_ptr(), ld, n, f_na.data_ptr())
    torch.cuda.synchronize()
    return f_ref.cpu().numpy(), f_na.cpu().numpy()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize(
    "obj,d,scale,rotated",
    [(1, 100, 1.0, True), (2, 37, 0.5, True), (3, 130, 1.0, True), (0, 10, 1.0, False), (1, 1, 2.0, True)],
)
def test_noalloc_equals_de_eval_two_calls(prec, obj, d, scale, rotated):
    torch = _need_gpu()
    o = problems.shift(d, seed=4) if rotated else None
    M = problems.rotation(d, seed=4) if rotated else None
    cfg = capi.make_config(64, d, objective=obj, scale=scale, shift=o, rot=M, precision=prec, max_generations=1)
    h = capi.de_init(cfg)
    try:
        od = None if o is None else torch.from_numpy(o).cuda()
        Md = None if M is None else torch.from_numpy(np.ascontiguousarray(M)).cuda()
        for call, (n, seed) in enumerate([(300, 11), (77, 12)]):
            X = problems.population(n, d, seed=seed)
            if o is not None:  # some rows near the optimum, where the terms are small
                X[:20] = o + np.random.default_rng(seed).normal(size=(20, d)) * 1e-3
            f_ref, f_na = _both(torch, h, prec, obj, d, scale, od, Md, X, ld=d + 3)
            assert np.array_equal(f_ref, f_na), f"call {call}: max diff {np.nanmax(np.abs(f_ref - f_na))}"
            oo = np.zeros(d) if o is None else o
            MM = np.eye(d) if M is None else M
            fo, sabs = oracle.evaluate(obj, X, oo, MM, scale=scale)
            err = np.abs(f_na - fo) / (np.abs(fo) + sabs)
            assert err.max() <= REL_SPLIT[prec], (call, err.max())
    finally:
        capi.de_destroy(h)


@pytest.mark.parametrize("prec", PRECS)
def test_noalloc_size_limit(prec):
    torch = _need_gpu()
    d, obj = 100, 1
    o = problems.shift(d, seed=6)
    M = problems.rotation(d, seed=6)
    nmax = MAX_ROWS_D100[prec]
    cfg = capi.make_config(64, d, objective=obj, shift=o, rot=M, precision=prec, max_generations=1)
    h = capi.de_init(cfg)
    try:
        od = torch.from_numpy(o).cuda()
        Md = torch.from_numpy(np.ascontiguousarray(M)).cuda()
        X = problems.population(nmax + 1, d, seed=7)
        # the largest n that fits is accepted and matches de_eval
        f_ref, f_na = _both(torch, h, prec, obj, d, 1.0, od, Md, X[:nmax], ld=d)
        assert np.array_equal(f_ref, f_na)
        # one row more is rejected before any launch: f stays untouched
        xd = torch.from_numpy(X).cuda()
        f = torch.full((nmax + 1,), -7.0, dtype=torch.float64, device="cuda")
        with pytest.raises(capi.DEError) as ei:
            capi.de_eval_noalloc(prec, obj, d, 1.0, od.data_ptr(), Md.data_ptr(), xd.data_ptr(), d, nmax + 1,
                                 f.data_ptr())
        torch.cuda.synchronize()
        assert ei.value.status == capi.DE_ERR_INVALID_ARG
        assert f"at most {nmax} rows" in str(ei.value)
        assert bool((f == -7.0).all())
    finally:
        capi.de_destroy(h)


# largest n per call at d = 1000 (4 N tiles of M) and largest d per precision
# for the 16 MiB scratch (stated in de.h)
MAX_ROWS_D1000 = {capi.DE_PREC_BF16X3: 3072, capi.DE_PREC_TF32X3: 1024}
MAX_D = {capi.DE_PREC_BF16X3: 1920, capi.DE_PREC_TF32X3: 1280}


@pytest.mark.parametrize("prec", PRECS)
def test_noalloc_d1000_at_the_row_limit_two_calls(prec):
    """d = 1000: M spans four 256-wide N tiles, which the kernel loops over.
    The first call takes the largest n that fits, the second a ragged n;
    both equal de_eval bit for bit."""
    torch = _need_gpu()
    d, obj = 1000, 1
    o, M = problems.shift(d, seed=12), problems.rotation(d, seed=12)
    cfg = capi.make_config(64, d, objective=obj, shift=o, rot=M, precision=prec, max_generations=1)
    h = capi.de_init(cfg)
    try:
        od = torch.from_numpy(o).cuda()
        Md = torch.from_numpy(np.ascontiguousarray(M)).cuda()
        nmax = MAX_ROWS_D1000[prec]
        for call, (n, seed) in enumerate([(nmax, 13), (nmax - 77, 14)]):
            X = problems.population(n, d, seed=seed)
            X[:8] = o + np.random.default_rng(seed).normal(size=(8, d)) * 1e-3
            f_ref, f_na = _both(torch, h, prec, obj, d, 1.0, od, Md, X, ld=d)
            assert np.array_equal(f_ref, f_na), f"call {call}"
            fo, sabs = oracle.evaluate(obj, X[:64], o, M)
            err = np.abs(f_na[:64] - fo) / (np.abs(fo) + sabs)
            assert err.max() <= REL_SPLIT[prec], (call, err.max())
        # one row more than fits is rejected
        X = torch.zeros((nmax + 1, d), dtype=torch.float64, device="cuda")
        f = torch.zeros(nmax + 1, dtype=torch.float64, device="cuda")
        with pytest.raises(capi.DEError) as ei:
            capi.de_eval_noalloc(prec, obj, d, 1.0, od.data_ptr(), Md.data_ptr(), X.data_ptr(), d, nmax + 1,
                                 f.data_ptr())
        assert ei.value.status == capi.DE_ERR_INVALID_ARG and f"at most {nmax} rows" in str(ei.value)
    finally:
        capi.de_destroy(h)


@pytest.mark.parametrize("prec", PRECS)
def test_noalloc_largest_d(prec):
    """The largest d whose split M fits the scratch is accepted (one tile,
    equal to de_eval); one more is rejected with the limit in the message."""
    torch = _need_gpu()
    d, obj, n = MAX_D[prec], 0, 128
    o, M = problems.shift(d, seed=15), problems.rotation(d, seed=15)
    od = torch.from_numpy(o).cuda()
    Md = torch.from_numpy(np.ascontiguousarray(M)).cuda()
    h = capi.de_init(capi.make_config(8, d, objective=obj, shift=o, rot=M, precision=prec, max_generations=1))
    try:
        X = problems.population(n, d, seed=16)
        f_ref, f_na = _both(torch, h, prec, obj, d, 1.0, od, Md, X, ld=d)
        assert np.array_equal(f_ref, f_na)
    finally:
        capi.de_destroy(h)
    d1 = d + 1
    X = torch.zeros((4, d1), dtype=torch.float64, device="cuda")
    f = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(capi.DEError) as ei:
        capi.de_eval_noalloc(prec, obj, d1, 1.0, None, None, X.data_ptr(), d1, 4, f.data_ptr())
    assert ei.value.status == capi.DE_ERR_INVALID_ARG
    assert f"the largest d is {d}" in str(ei.value)


def test_noalloc_allocates_nothing():
    """After the first call (one-time set-up), a call leaves the device's free
    memory unchanged."""
    torch = _need_gpu()
    d, obj, n = 100, 1, 1000
    o = torch.from_numpy(problems.shift(d, seed=8)).cuda()
    M = torch.from_numpy(np.ascontiguousarray(problems.rotation(d, seed=8))).cuda()
    X = torch.from_numpy(problems.population(n, d, seed=9)).cuda()
    f1 = torch.zeros(n, dtype=torch.float64, device="cuda")
    f2 = torch.zeros(n, dtype=torch.float64, device="cuda")
    for prec in PRECS:
        capi.de_eval_noalloc(prec, obj, d, 1.0, o.data_ptr(), M.data_ptr(), X.data_ptr(), d, n, f1.data_ptr())
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for prec in PRECS:
        capi.de_eval_noalloc(prec, obj, d, 1.0, o.data_ptr(), M.data_ptr(), X.data_ptr(), d, n, f2.data_ptr())
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    # both loops ended with the TF32X3 call on the same inputs
    assert torch.equal(f1, f2)


def test_noalloc_rejects_bad_arguments():
    torch = _need_gpu()
    d = 10
    X = torch.zeros((4, d), dtype=torch.float64, device="cuda")
    f = torch.zeros(4, dtype=torch.float64, device="cuda")
    host = np.zeros((4, d))
    with pytest.raises(capi.DEError) as ei:  # FP64 needs no scratch
        capi.de_eval_noalloc(capi.DE_PREC_FP64, 1, d, 1.0, None, None, X.data_ptr(), d, 4, f.data_ptr())
    assert ei.value.status == capi.DE_ERR_UNSUPPORTED
    with pytest.raises(capi.DEError) as ei:  # host memory is not device memory
        capi.de_eval_noalloc(capi.DE_PREC_BF16X3, 1, d, 1.0, None, None, host.ctypes.data, d, 4, f.data_ptr())
    assert ei.value.status == capi.DE_ERR_INVALID_ARG
    with pytest.raises(capi.DEError) as ei:  # ld < d
        capi.de_eval_noalloc(capi.DE_PREC_BF16X3, 1, d, 1.0, None, None, X.data_ptr(), d - 1, 4, f.data_ptr())
    assert ei.value.status == capi.DE_ERR_INVALID_ARG
