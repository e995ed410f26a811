"""Fitness error of every precision against the FP64 oracle, per objective
and dimension, in two measures:

  plain   |f_gpu - f_oracle| / |f_oracle|
  scaled  |f_gpu - f_oracle| / (|f_oracle| + S)   (S: the oracle's tolerance scale)

at uniform random points of [-100, 100]^D and at points 1e-3 and 1e-8 from
the optimum o (Sec. 7.3.1 objectives; the 1e-8 stopping target of Sec. 7.3.4
sits in the second group).  Asserted:
  * scaled <= 1e-12 (FP64), 1e-5 (BF16X3), 1e-6 (TF32X3) everywhere;
  * plain  <= 1e-12 (FP64), 1e-4 (BF16X3) and 3e-5 (TF32X3) at random
    points, where f is far from 0.  Near the optimum the plain measure is reported, not bounded:
    there even the correctly rounded FP64 evaluation in the written order
    misses 1e-12 (pinned in tests/test_oracle_tolerance.py).
Each case prints one line (run pytest with -s to see the table).
"""
import numpy as np
import pytest

import oracle
from paper_2405_16551_gb300 import capi, problems

pytestmark = pytest.mark.gpu

SCALED = {capi.DE_PREC_FP64: 1e-12, capi.DE_PREC_BF16X3: 1e-5, capi.DE_PREC_TF32X3: 1e-6}
# plain relative error at random points: BF16X3 keeps 16 bits of y and of M
# (bf16 high + low parts, the low x low product dropped), about 2^-16 per
# product; TF32X3 keeps 22 bits, and at D = 1000 the FP32 accumulation of the
# 1000 products dominates
PLAIN_RANDOM = {capi.DE_PREC_FP64: 1e-12, capi.DE_PREC_BF16X3: 1e-4, capi.DE_PREC_TF32X3: 3e-5}
NAMES = {capi.DE_PREC_FP64: "FP64", capi.DE_PREC_BF16X3: "BF16X3", capi.DE_PREC_TF32X3: "TF32X3"}
OBJ = {0: "sphere", 1: "rastrigin", 2: "rosenbrock", 3: "ackley"}


def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("prec", [capi.DE_PREC_FP64, capi.DE_PREC_BF16X3, capi.DE_PREC_TF32X3])
@pytest.mark.parametrize("d", [10, 100, 1000])
@pytest.mark.parametrize("obj", [0, 1, 2, 3])
def test_fitness_error_per_objective(prec, d, obj):
    torch = _need_gpu()
    if obj == 2 and prec != capi.DE_PREC_FP64 and d > 256:
        pytest.skip("split-precision Rosenbrock is limited to d <= 256")
    n = 256
    o, M = problems.shift(d, seed=50 + d), problems.rotation(d, seed=50 + d)
    rng = np.random.default_rng(d + obj)
    groups = {"random": problems.population(n, d, seed=60 + d),
              "1e-3 from o": o + 1e-3 * rng.uniform(-1, 1, (n, d)),
              "1e-8 from o": o + 1e-8 * rng.uniform(-1, 1, (n, d))}
    h = capi.de_init(capi.make_config(64, d, objective=obj, shift=o, rot=M, precision=prec, max_generations=1))
    try:
        for name, X in groups.items():
            xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
            fd = torch.zeros(n, dtype=torch.float64, device="cuda")
            capi.de_eval(h, 0, xd.data_ptr(), d, n, fd.data_ptr())
            torch.cuda.synchronize()
            f = fd.cpu().numpy()
            fo, S = oracle.evaluate(obj, X, o, M)
            err = np.abs(f - fo)
            scaled = float((err / (np.abs(fo) + S)).max())
            nz = np.abs(fo) > 0
            plain = float((err[nz] / np.abs(fo[nz])).max()) if nz.any() else 0.0
            print(f"ACCURACY {NAMES[prec]:6s} {OBJ[obj]:10s} d={d:5d} {name:12s} plain={plain:.2e} "
                  f"scaled={scaled:.2e} median|f|={float(np.median(np.abs(fo))):.3e}")
            assert scaled <= SCALED[prec], (name, scaled)
            if name == "random":
                assert plain <= PLAIN_RANDOM[prec], (name, plain)
    finally:
        capi.de_destroy(h)
