"""Seeded synthetic problem data (shift vectors, rotation matrices, batch shapes,
hidden ODE parameters).

The benchmark of arXiv 2405.16551 (Sec. 7.3.1) supplies, per function, a shift
vector o with entries in [-80, 80] and a rotation matrix M, both read from the
CEC'14/'17 input files.  Those files are not available here, so this module
draws stand-ins of the same shapes from numpy's seeded generators:

* ``shift(d, seed, run_id)``: o ~ U[-80, 80]^d;
* ``rotation(d, seed, run_id)``: the orthogonal factor of the QR decomposition of
  a standard Gaussian d x d matrix, with column signs fixed so that R has a
  positive diagonal (Haar-distributed orthogonal matrix, Mezzadri 2007);
* ``batch_shapes(nruns, seed)``: per-run (NP, D, objective) for the batched
  workload: D from {10, 30, 50, 100}, NP uniform in {50..1000}, one of four
  objectives;
* ``ode_hidden(seed)``: the hidden parameter vector whose trajectory the ODE
  objective fits;
* ``permutation(d, seed, run_id)``: the shuffle of a hybrid function
  (Sec. 7.3.2), a uniform random permutation of 0..d-1;
* ``suite(objective, d, seed)``: the data of one function of the proposed
  benchmark (Table 2): n shift vectors and n rotations (n = 3, 4, 5 for the
  composition functions, 1 otherwise) and the permutation.

This module holds no step of the DE method itself: it only makes the data a
problem is defined by, which both the CUDA library and the CPU oracle take as
input.  It depends on numpy alone and imports nothing from the library.
"""
from __future__ import annotations

import numpy as np

SPHERE, RASTRIGIN, ROSENBROCK, ACKLEY = 0, 1, 2, 3
OBJECTIVE_NAMES = {SPHERE: "sphere", RASTRIGIN: "rastrigin", ROSENBROCK: "rosenbrock", ACKLEY: "ackley"}

_TAG_SHIFT, _TAG_ROT, _TAG_BATCH, _TAG_ODE, _TAG_POP, _TAG_PERM = 11, 12, 13, 14, 15, 16

# the proposed benchmark (Table 2): function number -> objective id of the
# library, and the number of (shift, rotation) pairs a composition function takes
ZAKHAROV, SCHWEFEL = 5, 6
HYBRID1, HYBRID2, HYBRID3, COMPOSITION1, COMPOSITION2, COMPOSITION3 = 15, 16, 17, 18, 19, 20
SUITE = {1: ZAKHAROV, 2: ROSENBROCK, 3: RASTRIGIN, 4: SCHWEFEL, 5: HYBRID1, 6: HYBRID2, 7: HYBRID3,
         8: COMPOSITION1, 9: COMPOSITION2, 10: COMPOSITION3}
_COMPONENTS = {COMPOSITION1: 3, COMPOSITION2: 4, COMPOSITION3: 5}
# search-domain scale of the suite's stand-alone basic functions (the
# Rosenbrock, Rastrigin and modified Schwefel functions map [-100, 100] onto
# their customary domains); 1 for the others
SUITE_SCALE = {ROSENBROCK: 2.048 / 100.0, RASTRIGIN: 5.12 / 100.0, SCHWEFEL: 1000.0 / 100.0}


def _rng(seed: int, run_id: int, tag: int) -> np.random.Generator:
    return np.random.default_rng([int(seed) & 0xFFFFFFFFFFFFFFFF, int(run_id), int(tag)])


def shift(d: int, seed: int = 1, run_id: int = 0, lo: float = -80.0, hi: float = 80.0) -> np.ndarray:
    """Shift vector o ~ U[lo, hi]^d (Sec. 7.3.1 places the optimum in [-80, 80])."""
    return _rng(seed, run_id, _TAG_SHIFT).uniform(lo, hi, size=d)


def rotation(d: int, seed: int = 1, run_id: int = 0) -> np.ndarray:
    """Row-major orthogonal d x d matrix M (z = M y, Sec. 7.3.1)."""
    g = _rng(seed, run_id, _TAG_ROT).standard_normal((d, d))
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return np.ascontiguousarray(q * s[None, :])


def batch_shapes(nruns: int, seed: int = 1, dims=(10, 30, 50, 100), np_lo: int = 50, np_hi: int = 1000):
    """Per-run (np, d, objective) for a batch of independent runs."""
    g = _rng(seed, 0, _TAG_BATCH)
    d = g.choice(np.asarray(dims), size=nruns)
    n = g.integers(np_lo, np_hi + 1, size=nruns)
    obj = g.integers(0, 4, size=nruns)
    return [(int(n[r]), int(d[r]), int(obj[r])) for r in range(nruns)]


def ode_hidden(seed: int = 1, d: int = 20) -> np.ndarray:
    """Hidden parameter vector in [-100, 100]^d for the ODE fitting objective."""
    return _rng(seed, 0, _TAG_ODE).uniform(-100.0, 100.0, size=d)


def population(np_: int, d: int, seed: int = 1, lo: float = -100.0, hi: float = 100.0) -> np.ndarray:
    """A population drawn uniformly in [lo, hi)^d, for tests that feed the same
    population to both sides of a comparison."""
    return _rng(seed, 0, _TAG_POP).uniform(lo, hi, size=(np_, d))


def permutation(d: int, seed: int = 1, run_id: int = 0) -> np.ndarray:
    """Uniform random permutation of 0..d-1 (int32), the shuffle of a hybrid function."""
    return _rng(seed, run_id, _TAG_PERM).permutation(d).astype(np.int32)


def suite(objective: int, d: int, seed: int = 1) -> dict:
    """Shift (n x d), rotation (n x d x d) and permutation (d; hybrid functions
    only, else None) of one function of the proposed benchmark; n = 1 except
    for the composition functions.  For n = 1 the shift is a vector and the
    rotation a matrix."""
    n = _COMPONENTS.get(objective, 1)
    o = np.stack([shift(d, seed=seed, run_id=c) for c in range(n)])
    M = np.stack([rotation(d, seed=seed, run_id=c) for c in range(n)])
    if n == 1:
        o, M = o[0], M[0]
    perm = permutation(d, seed=seed) if objective in (HYBRID1, HYBRID2, HYBRID3) else None
    return {"shift": o, "rot": M, "perm": perm, "scale": SUITE_SCALE.get(objective, 1.0)}
