"""GPU surrogate network (BF16 tcgen05 products, FP32 accumulation) against
the FP64 CPU oracle, through the C ABI.

Forward: |y_gpu - y| <= 2^-5 * S_y, where S_y is the output of the same
network with every weight, bias and input replaced by its absolute value.
Four roundings to BF16 (input, W1, hidden activations, W2), each at most
2^-8 relative, bound the error of every product term by about 2^-6 of its
magnitude; the margin doubles that.
Gradients: BF16 operands in every product give percent-level relative
errors per element.  The test bounds the normwise relative error of each
parameter block (0.05) and asks for a cosine similarity near 1.
Adam: with every minibatch row identical, the sampled minibatch has the same
gradient as the ordered one; one GPU step must equal the oracle's Adam
update of that gradient up to FP32 rounding.
"""
import numpy as np
import pytest

import oracle
from paper_2405_16551_gb300 import capi, problems

pytestmark = pytest.mark.gpu


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _abs_params(p):
    return {k: np.abs(v) for k, v in p.items()}


def _oracle_params(params):
    p = capi.mlp_unpack(params)
    # the oracle takes x itself; the network sees x / 100
    p["W1"] = p["W1"] / 100.0
    return p


@pytest.mark.parametrize("seed,n", [(1, 300), (2, 128), (3, 1), (4, 1000)])
def test_mlp_forward_matches_oracle(seed, n):
    torch = _need_gpu()
    m = capi.de_mlp_create(seed)
    try:
        params = capi.de_mlp_get_params(m)
        if seed == 2:  # nonzero biases everywhere
            g = np.random.default_rng(seed)
            d = capi.mlp_unpack(params)
            for k in ("b1", "b2", "b3"):
                d[k] = g.normal(size=d[k].shape) * 0.3
            params = capi.mlp_pack(d)
            capi.de_mlp_set_params(m, params)
        X = problems.population(n, 20, seed=seed)
        xd = torch.from_numpy(X).cuda()
        yd = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
        capi.de_mlp_forward(m, xd.data_ptr(), 20, n, yd.data_ptr())
        torch.cuda.synchronize()
    finally:
        capi.de_mlp_destroy(m)
    y = yd.cpu().numpy().astype(np.float64)
    p = _oracle_params(params)
    yo = oracle.mlp_forward(p, X)
    sy = oracle.mlp_forward(_abs_params(p), np.abs(X))
    err = np.abs(y - yo)
    assert np.all(err <= 2.0 ** -5 * sy + 1e-6), float(np.max(err / sy))
    # typical error far below the bound
    assert np.sqrt(np.mean((err / sy) ** 2)) < 2.0 ** -8


def test_mlp_gradient_matches_oracle():
    torch = _need_gpu()
    m = capi.de_mlp_create(7)
    try:
        params = capi.de_mlp_get_params(m)
        X = problems.population(256, 20, seed=8)
        t = np.random.default_rng(9).normal(size=256).astype(np.float32)
        xd = torch.from_numpy(X).cuda()
        td = torch.from_numpy(t).cuda()
        g, loss = capi.de_mlp_grad(m, xd.data_ptr(), 20, td.data_ptr())
        # the gradient call leaves the parameters as they were
        assert np.array_equal(capi.de_mlp_get_params(m), params)
    finally:
        capi.de_mlp_destroy(m)
    p = _oracle_params(params)
    lo, go = oracle.mlp_loss_grad(p, X, t.astype(np.float64))
    go["W1"] = go["W1"] / 100.0  # gradient with respect to the network's own W1 (input x / 100)
    gg = capi.mlp_unpack(g)
    assert loss == pytest.approx(lo, rel=2e-2)
    for k in oracle.MLP_KEYS:
        a, b = gg[k].ravel(), go[k].ravel()
        nb = np.linalg.norm(b)
        assert np.linalg.norm(a - b) <= 0.05 * nb + 1e-7, (k, np.linalg.norm(a - b) / nb)
        if nb > 0:
            assert np.dot(a, b) / (np.linalg.norm(a) * nb) > 0.998, k


def test_mlp_adam_step_matches_oracle():
    torch = _need_gpu()
    m = capi.de_mlp_create(11)
    try:
        p0 = capi.de_mlp_get_params(m)
        row = problems.population(1, 20, seed=12)
        X = np.repeat(row, 256, axis=0)
        t = np.full(256, 0.7, dtype=np.float32)
        xd = torch.from_numpy(X).cuda()
        td = torch.from_numpy(t).cuda()
        g, _ = capi.de_mlp_grad(m, xd.data_ptr(), 20, td.data_ptr())
        lr = 1e-3
        capi.de_mlp_train(m, xd.data_ptr(), 20, td.data_ptr(), 256, 1, lr)
        p1 = capi.de_mlp_get_params(m)
    finally:
        capi.de_mlp_destroy(m)
    w = p0.astype(np.float64)
    mo = np.zeros_like(w)
    vo = np.zeros_like(w)
    oracle.adam(w, g.astype(np.float64), mo, vo, 1, lr=lr)
    tol = 2.0 ** -22 * (np.abs(w) + lr) + 1e-12
    assert np.all(np.abs(p1 - w) <= tol), float(np.max(np.abs(p1 - w) - tol))
    moved = np.abs(g) > 1e-4
    assert moved.sum() > 1000
    assert np.allclose(np.abs(p1 - p0)[moved], lr, rtol=1e-3)


def test_mlp_training_fits_a_function():
    """Adam on 4096 rows of a smooth target: the loss falls by 10x."""
    torch = _need_gpu()
    X = problems.population(4096, 20, seed=13)
    t = (np.sin(X[:, 0] / 30.0) + (X[:, 1] / 100.0) * (X[:, 2] / 100.0) + 0.5 * (X[:, 3] / 100.0) ** 2)
    t = ((t - t.mean()) / t.std()).astype(np.float32)
    m = capi.de_mlp_create(14)
    try:
        xd = torch.from_numpy(X).cuda()
        td = torch.from_numpy(t).cuda()
        l0 = capi.de_mlp_grad(m, xd.data_ptr(), 20, td.data_ptr())[1]
        capi.de_mlp_train(m, xd.data_ptr(), 20, td.data_ptr(), 4096, 600, 1e-3)
        l1 = capi.de_mlp_grad(m, xd.data_ptr(), 20, td.data_ptr())[1]
        yd = torch.zeros(4096, dtype=torch.float32, device="cuda")
        capi.de_mlp_forward(m, xd.data_ptr(), 20, 4096, yd.data_ptr())
        torch.cuda.synchronize()
    finally:
        capi.de_mlp_destroy(m)
    assert l1 < 0.1 * l0, (l0, l1)
    y = yd.cpu().numpy()
    assert np.mean((y - t) ** 2) < 0.1


def test_mlp_rejects_bad_arguments():
    _need_gpu()
    m = capi.de_mlp_create(1)
    try:
        with pytest.raises(capi.DEError):
            capi.de_mlp_forward(m, 0, 20, 4, 0)
        bad = np.zeros(capi.DE_MLP_PARAMS, dtype=np.float32)
        bad[5] = np.nan
        with pytest.raises(capi.DEError):
            capi.de_mlp_set_params(m, bad)
    finally:
        capi.de_mlp_destroy(m)
