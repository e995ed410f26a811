"""Pins of the oracle's benchmark suite (Sec. 7.3, Table 2): the basic
functions, the hybrid split (Sec. 7.3.2) and the composition weights
(Sec. 7.3.3), against optima, special points with closed forms, identities
between independently written functions, and the plain weight formula.
CPU only."""
import math

import numpy as np
import pytest

import oracle
from paper_2405_16551_gb300 import problems

BASIC = [oracle.SPHERE, oracle.RASTRIGIN, oracle.ROSENBROCK, oracle.ACKLEY, oracle.ZAKHAROV, oracle.SCHWEFEL,
         oracle.BENT_CIGAR, oracle.HGBAT, oracle.SCHAFFER_F6, oracle.KATSUURA, oracle.HAPPYCAT,
         oracle.GRIEWANK_ROSENBROCK, oracle.ELLIPTIC, oracle.GRIEWANK]
SUITE = [oracle.ZAKHAROV, oracle.ROSENBROCK, oracle.RASTRIGIN, oracle.SCHWEFEL, oracle.HYBRID1, oracle.HYBRID2,
         oracle.HYBRID3, oracle.COMPOSITION1, oracle.COMPOSITION2, oracle.COMPOSITION3]


@pytest.mark.parametrize("fn", BASIC)
@pytest.mark.parametrize("n", [1, 2, 10, 37])
def test_basic_functions_vanish_at_the_optimum(fn, n):
    f, _ = oracle.basic(fn, np.zeros(n))
    assert abs(f) <= 1e-12


@pytest.mark.parametrize("fn", BASIC)
def test_basic_functions_are_nonnegative(fn):
    rng = np.random.default_rng(fn)
    for n in (1, 3, 10, 50):
        for _ in range(50):
            z = rng.uniform(-5, 5, n) * rng.choice([0.01, 1.0, 20.0])
            f, S = oracle.basic(fn, z)
            assert f >= -1e-12 * (1 + S), (fn, n, f)


def test_special_points():
    e = np.eye(5)
    assert oracle.basic(oracle.BENT_CIGAR, e[0])[0] == 1.0
    assert oracle.basic(oracle.BENT_CIGAR, e[3])[0] == 1e6
    assert oracle.basic(oracle.ELLIPTIC, e[0])[0] == 1.0
    assert oracle.basic(oracle.ELLIPTIC, e[2])[0] == pytest.approx(1e3, rel=1e-15)
    assert oracle.basic(oracle.ELLIPTIC, e[4])[0] == pytest.approx(1e6, rel=1e-15)
    # Zakharov in 2-D at the unit vectors: 1 + (i/2)^2 + (i/2)^4
    assert oracle.basic(oracle.ZAKHAROV, [1.0, 0.0])[0] == 1.3125
    assert oracle.basic(oracle.ZAKHAROV, [0.0, 1.0])[0] == 3.0
    # HGBat and HappyCat at x = z - 1 = 0
    assert oracle.basic(oracle.HGBAT, np.ones(7))[0] == 0.5
    assert oracle.basic(oracle.HAPPYCAT, np.ones(16))[0] == pytest.approx(2.5, rel=1e-15)
    # Katsuura vanishes wherever every 2^j z_i is an integer, and at z = 2^-40
    # (all 32 fractional parts equal 2^j z) it is 10 ((1 + 32 z)^10 - 1) in 1-D
    assert oracle.basic(oracle.KATSUURA, np.array([3.0, -0.5, 1.5, 7.0]))[0] == 0.0
    # at z = 1/4 only the j = 1 term is nonzero: 0.5 / 2
    assert oracle.basic(oracle.KATSUURA, [0.25])[0] == pytest.approx(10 * (1.25 ** 10 - 1), rel=1e-14)
    t = 2.0 ** -40
    assert oracle.basic(oracle.KATSUURA, [t])[0] == pytest.approx(10 * ((1 + 32 * t) ** 10 - 1), rel=1e-9)
    # Schaffer F6 pair at radius pi: sin r = 0
    g = 0.5 - 0.5 / (1 + 0.001 * math.pi ** 2) ** 2
    assert oracle.basic(oracle.SCHAFFER_F6, [math.pi, 0.0])[0] == pytest.approx(2 * g, rel=1e-14)
    # Griewank where every cosine is 1: only the quadratic part remains
    z = np.array([2 * math.pi * math.sqrt(i + 1) * m for i, m in enumerate([1, -2, 3, 1])])
    assert oracle.basic(oracle.GRIEWANK, z)[0] == pytest.approx(float(np.sum(z * z)) / 4000, rel=1e-12)


def test_schwefel_optimum_location_and_folding():
    c0 = 420.9687462275036
    # moving off the optimum in any coordinate increases f
    for dz in (-1.0, -0.01, 0.01, 1.0):
        assert oracle.basic(oracle.SCHWEFEL, [0.0, dz, 0.0])[0] > 0.0
    # continuous at t = +-500 where the folding starts
    for edge in (500.0, -500.0):
        a = oracle.basic(oracle.SCHWEFEL, [edge - 1e-9 - c0])[0]
        b = oracle.basic(oracle.SCHWEFEL, [edge + 1e-9 - c0])[0]
        assert abs(a - b) < 1e-6
    # folding: t and t - 500 k (k >= 1 beyond the box) share the sine part
    t = 777.0
    n = 1
    inner = oracle.basic(oracle.SCHWEFEL, [277.0 - c0])[0]
    outer = oracle.basic(oracle.SCHWEFEL, [t - c0])[0]
    fmax = 418.9828872724338
    # outer = fmax - [(500 - 277) sin sqrt(223) - 277^2 / 1e4]; inner = fmax - 277 sin sqrt(277)
    assert outer == pytest.approx(fmax - (223 * math.sin(math.sqrt(223)) - 277.0 ** 2 / 1e4 / n), rel=1e-13)
    assert inner == pytest.approx(fmax - 277 * math.sin(math.sqrt(277)), rel=1e-13)


def test_griewank_rosenbrock_is_griewank_of_rosenbrock_pairs():
    """The expanded Griewank-plus-Rosenbrock equals the 1-D Griewank function
    applied to the 2-D Rosenbrock function of each cyclic pair (two other,
    separately written basic functions)."""
    rng = np.random.default_rng(3)
    for n in (1, 2, 5, 12):
        z = rng.uniform(-1.5, 1.5, n)
        want = 0.0
        for k in range(n):
            r, _ = oracle.basic(oracle.ROSENBROCK, [z[k], z[(k + 1) % n]])
            want += oracle.basic(oracle.GRIEWANK, [r])[0]
        assert oracle.basic(oracle.GRIEWANK_ROSENBROCK, z)[0] == pytest.approx(want, rel=1e-13, abs=1e-13)


@pytest.mark.parametrize("fn", [oracle.SPHERE, oracle.RASTRIGIN, oracle.ROSENBROCK, oracle.ACKLEY])
def test_suite_copies_of_the_classic_functions_match_the_objectives(fn):
    """or_basic's sphere, Rastrigin, Rosenbrock and Ackley (used inside the
    hybrid and composition functions) equal the separately written objectives."""
    rng = np.random.default_rng(fn)
    for n in (1, 2, 17):
        z = rng.uniform(-3, 3, n)
        f0, _ = oracle.objective(fn, z)
        assert oracle.basic(fn, z)[0] == pytest.approx(f0, rel=1e-14, abs=1e-14)


def test_hybrid_segments():
    # ceil(p d) for the first parts, the rest for the last
    assert list(oracle.hybrid_segments(oracle.HYBRID1, 10)) == [0, 3, 6, 10]
    assert list(oracle.hybrid_segments(oracle.HYBRID1, 30)) == [0, 9, 18, 30]
    assert list(oracle.hybrid_segments(oracle.HYBRID2, 50)) == [0, 10, 20, 35, 50]
    assert list(oracle.hybrid_segments(oracle.HYBRID3, 10)) == [0, 3, 5, 7, 8, 10]
    assert list(oracle.hybrid_segments(oracle.HYBRID3, 100)) == [0, 30, 50, 70, 80, 100]
    assert oracle.hybrid_segments(oracle.HYBRID3, 6) is None
    assert oracle.hybrid_segments(oracle.COMPOSITION1, 10) is None


@pytest.mark.parametrize("obj", [oracle.HYBRID1, oracle.HYBRID2, oracle.HYBRID3])
def test_hybrid_is_the_sum_of_its_parts(obj):
    d = 30
    rng = np.random.default_rng(obj)
    o = problems.shift(d, seed=obj)
    M = problems.rotation(d, seed=obj)
    perm = rng.permutation(d).astype(np.int32)
    x = rng.uniform(-100, 100, d)
    f, _ = oracle.objective(obj, x, o, M, perm=perm)
    z = M @ (x - o)
    zp = z[perm]
    seg = oracle.hybrid_segments(obj, d)
    fns = {oracle.HYBRID1: [oracle.BENT_CIGAR, oracle.HGBAT, oracle.RASTRIGIN],
           oracle.HYBRID2: [oracle.SCHAFFER_F6, oracle.HGBAT, oracle.ROSENBROCK, oracle.SCHWEFEL],
           oracle.HYBRID3: [oracle.KATSUURA, oracle.HAPPYCAT, oracle.GRIEWANK_ROSENBROCK, oracle.SCHWEFEL,
                            oracle.ACKLEY]}[obj]
    want = sum(oracle.basic(fn, oracle.domain_scale(fn) * zp[seg[c]:seg[c + 1]])[0] for c, fn in enumerate(fns))
    assert f == pytest.approx(want, rel=1e-9)
    # at x = o every part sits at its optimum
    f0, _ = oracle.objective(obj, o, o, M, perm=perm)
    assert abs(f0) <= 1e-9


def _composition_data(obj, d, seed):
    n = oracle.suite_components(obj)
    o = np.stack([problems.shift(d, seed=seed, run_id=c) for c in range(n)])
    M = np.stack([problems.rotation(d, seed=seed, run_id=c) for c in range(n)])
    return o, M


COMP = {oracle.COMPOSITION1: ([oracle.RASTRIGIN, oracle.GRIEWANK, oracle.SCHWEFEL], [10, 20, 30], [1, 10, 1],
                              [0, 100, 200]),
        oracle.COMPOSITION2: ([oracle.ACKLEY, oracle.ELLIPTIC, oracle.GRIEWANK, oracle.RASTRIGIN], [10, 20, 30, 40],
                              [10, 1e-6, 10, 1], [0, 100, 200, 300]),
        oracle.COMPOSITION3: ([oracle.SCHAFFER_F6, oracle.SCHWEFEL, oracle.GRIEWANK, oracle.ROSENBROCK,
                               oracle.RASTRIGIN], [10, 20, 20, 30, 40], [0.005, 1, 10, 1, 10],
                              [0, 100, 200, 300, 400])}


@pytest.mark.parametrize("obj", list(COMP))
def test_composition_optima_carry_their_bias(obj):
    d = 20
    o, M = _composition_data(obj, d, 5)
    fns, sig, lam, bias = COMP[obj]
    for c in range(len(fns)):
        f, _ = oracle.objective(obj, o[c], o, M)
        assert f == pytest.approx(bias[c], abs=1e-9)
    # the global optimum (bias 0) is approached continuously
    f, _ = oracle.objective(obj, o[0] + 1e-7, o, M)
    assert 0 <= f < 1e-3


@pytest.mark.parametrize("obj", list(COMP))
def test_composition_matches_the_plain_weight_formula(obj):
    """Where no weight underflows, the logarithmic normalisation gives the
    paper's w_i / sum w_k."""
    d = 10
    o, M = _composition_data(obj, d, 9)
    fns, sig, lam, bias = COMP[obj]
    rng = np.random.default_rng(obj)
    for _ in range(20):
        c0 = rng.integers(len(fns))
        x = o[c0] + rng.normal(0, 8, d)
        g = [oracle.basic(fn, M[c] @ ((x - o[c]) * oracle.domain_scale(fn)))[0] for c, fn in enumerate(fns)]
        D = [float(np.sum((x - o[c]) ** 2)) for c in range(len(fns))]
        w = np.array([math.exp(-D[c] / (2 * d * sig[c] ** 2)) / math.sqrt(D[c]) for c in range(len(fns))])
        assert w.min() > 1e-300
        om = w / w.sum()
        want = float(sum(om[c] * (lam[c] * g[c] + bias[c]) for c in range(len(fns))))
        f, _ = oracle.objective(obj, x, o, M)
        assert f == pytest.approx(want, rel=1e-9)


@pytest.mark.parametrize("obj", SUITE)
def test_tolerance_scale_covers_input_perturbations(obj):
    """Relative perturbations of x of a few ulps move f by much less than
    1e-12 (|f| + S), so S is not too small to hold a correct evaluation in
    another rounding order."""
    d = 30
    rng = np.random.default_rng(100 + obj)
    if obj >= oracle.COMPOSITION1:
        o, M = _composition_data(obj, d, 3)
    else:
        o, M = problems.shift(d, seed=3), problems.rotation(d, seed=3)
    perm = rng.permutation(d).astype(np.int32)
    for _ in range(40):
        x = rng.uniform(-100, 100, d)
        f, S = oracle.objective(obj, x, o, M, perm=perm)
        xp = x * (1 + rng.choice([-1, 1], d) * 4e-16)
        fp, _ = oracle.objective(obj, xp, o, M, perm=perm)
        assert abs(fp - f) <= 1e-13 * (abs(f) + S), (obj, f, fp, S)
