"""GPU parity of the ODE fitting objective (FP64) against the CPU oracle.

The GPU integrates each chain with one IEEE operation per step of the same
stated order as the oracle, so trajectories agree bit for bit and f differs
only by the order of the final sum (tolerance rel * (|f| + S), rel = 1e-12).
f is exactly 0 at the hidden parameter vector.  One generation and a short
run follow the oracle's indices, masks, trials and decisions.  C ABI only.
"""
import numpy as np
import pytest

import oracle
from paper_2405_16551_gb300 import capi, problems

pytestmark = pytest.mark.gpu

REL64 = 1e-12
D = 20


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _cfg(np_, xh, **kw):
    return capi.make_config(np_, D, objective=capi.DE_OBJ_ODE, shift=xh, precision=capi.DE_PREC_FP64, **kw)


@pytest.mark.parametrize("seed", [1, 2])
def test_ode_eval_matches_oracle(seed):
    torch = _need_gpu()
    xh = problems.ode_hidden(seed)
    X = problems.population(70, D, seed=seed + 10)
    X[0] = xh
    X[1:6] = xh + np.random.default_rng(seed).normal(size=(5, D)) * np.array([1e-6, 1e-4, 1e-2, 1.0, 10.0])[:, None]
    h = capi.de_init(_cfg(32, xh, max_generations=1))
    try:
        xd = torch.from_numpy(X).cuda()
        fd = torch.full((len(X),), float("nan"), dtype=torch.float64, device="cuda")
        capi.de_eval(h, 0, xd.data_ptr(), D, len(X), fd.data_ptr())
        torch.cuda.synchronize()
    finally:
        capi.de_destroy(h)
    f = fd.cpu().numpy()
    fo, s = oracle.evaluate(capi.DE_OBJ_ODE, X, xh)
    assert f[0] == 0.0 and fo[0] == 0.0
    assert np.all(np.abs(f - fo) <= REL64 * (np.abs(fo) + s))
    # identical trajectories: only the summation order of f differs
    pos = fo > 0
    assert np.max(np.abs(f[pos] - fo[pos]) / fo[pos]) < 1e-13


def test_ode_init_population_and_best():
    _need_gpu()
    xh = problems.ode_hidden(3)
    h = capi.de_init(_cfg(48, xh, seed=9, max_generations=5))
    try:
        x, f = capi.de_get_population(h)
        b = capi.de_get_best(h)
    finally:
        capi.de_destroy(h)
    xo = oracle.init_population(48, D, -100.0, 100.0, seed=9)
    assert np.array_equal(x, xo)
    fo, s = oracle.evaluate(capi.DE_OBJ_ODE, xo, xh)
    assert np.all(np.abs(f - fo) <= REL64 * (np.abs(fo) + s))
    assert b["best_index"] == int(np.argmin(fo))


@pytest.mark.parametrize("np_,F,CR", [(48, 0.5, 0.9), (7, 0.8, 0.3), (4, 1.9, 1.0)])
def test_ode_one_generation_matches_oracle(np_, F, CR):
    _need_gpu()
    xh = problems.ode_hidden(4)
    X = problems.population(np_, D, seed=5)
    fX, _ = oracle.evaluate(capi.DE_OBJ_ODE, X, xh)
    cfg = _cfg(np_, xh, f=F, cr=CR, seed=11, max_generations=10**6, target_error=0.0, debug_capture=True)
    h = capi.de_init(cfg)
    try:
        capi.de_set_population(h, 0, X, fX)
        capi.de_set_generation(h, 0, 2)
        capi.de_step(h, 1)
        g = capi.de_get_debug(h)
        xn, fn = capi.de_get_population(h)
    finally:
        capi.de_destroy(h)
    r = oracle.step(X, fX, F, CR, -100.0, 100.0, capi.DE_OBJ_ODE, xh, None, seed=11, generation=3)
    assert np.array_equal(g["idx"], r["idx"])
    assert np.array_equal(g["mask"], r["mask"])
    assert np.array_equal(g["trial"], r["trial"])
    tol = REL64 * (np.abs(r["f_trial"]) + r["sabs_trial"])
    assert np.all(np.abs(g["f_trial"] - r["f_trial"]) <= tol)
    band = np.abs(r["f_trial"] - fX) <= tol
    assert np.array_equal(g["accept"][~band], r["accept"][~band])
    acc = g["accept"].astype(bool)
    assert np.array_equal(xn[acc], r["trial"][acc])
    assert np.array_equal(xn[~acc], X[~acc])


def test_ode_short_run_follows_oracle():
    """Ten generations of NP = 24 from the same seed: same population."""
    _need_gpu()
    xh = problems.ode_hidden(5)
    Xo, fo, go, evo, _ = oracle.run(24, D, 0.5, 0.9, -100, 100, capi.DE_OBJ_ODE, xh, None, seed=3,
                                 max_generations=10, target_error=0.0)
    h = capi.de_init(_cfg(24, xh, seed=3, max_generations=10, target_error=0.0))
    try:
        res = capi.de_run(h)[0]
        x, f = capi.de_get_population(h)
    finally:
        capi.de_destroy(h)
    assert res["generations"] == go == 10
    assert np.array_equal(x, Xo)
    assert np.allclose(f, fo, rtol=1e-13, atol=0)
