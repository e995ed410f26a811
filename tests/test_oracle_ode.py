"""Pins of the oracle's ODE fitting objective against facts that do not come
from the oracle itself: the exact solution of the linear chain (matrix
exponential), fourth-order convergence of RK4, conservation of the chain's
energy without damping and its decay with damping, the affine parameter map at
closed-form points, and f = 0 at the hidden parameters.  CPU only.

The chain (a reading; the paper motivates costly objectives in its Abstract
but defines none): unit masses, springs k_i to ground, dampers c_i, neighbour
springs of stiffness 1, both ends tied to walls, q(0) = e_1, p(0) = 0.
"""
import numpy as np
import pytest

import oracle
from paper_2405_16551_gb300 import problems

scipy_linalg = pytest.importorskip("scipy.linalg")

N = 10


def _system_matrix(k, c):
    """ds/dt = A s for s = (q, p), written from the equations of motion."""
    lap = 2.0 * np.eye(N) - np.eye(N, k=1) - np.eye(N, k=-1)  # fixed ends
    A = np.zeros((2 * N, 2 * N))
    A[:N, N:] = np.eye(N)
    A[N:, :N] = -np.diag(k) - lap
    A[N:, N:] = -np.diag(c)
    return A


def _exact_positions(k, c, times):
    A = _system_matrix(k, c)
    s0 = np.zeros(2 * N)
    s0[0] = 1.0
    return np.array([(scipy_linalg.expm(A * t) @ s0)[:N] for t in times])


def _energy(k, q, p):
    """Kinetic + ground springs + neighbour springs (walls at both ends)."""
    ext = np.concatenate([[0.0], q, [0.0]])
    return 0.5 * np.sum(p * p) + 0.5 * np.sum(k * q * q) + 0.5 * np.sum(np.diff(ext) ** 2)


def test_parameter_map_closed_form_points():
    x = np.concatenate([np.full(N, -100.0), np.full(N, 100.0)])
    k, c = oracle.ode_params(x)
    assert np.all(k == 0.5) and np.all(c == 0.5)
    x = np.concatenate([np.full(N, 100.0), np.full(N, -100.0)])
    k, c = oracle.ode_params(x)
    assert np.all(k == 5.0) and np.all(c == 0.01)
    k, c = oracle.ode_params(np.zeros(2 * N))
    assert np.allclose(k, 2.75, rtol=0, atol=1e-15) and np.allclose(c, 0.255, rtol=0, atol=1e-15)
    # oscillator i takes x_i and x_{10+i}
    x = np.zeros(2 * N)
    x[3] = 100.0
    x[N + 7] = -100.0
    k, c = oracle.ode_params(x)
    assert k[3] == 5.0 and c[7] == 0.01 and k[2] == k[4] and c[6] == c[8]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_rk4_matches_matrix_exponential(seed):
    rng = np.random.default_rng(seed)
    k = rng.uniform(0.5, 5.0, N)
    c = rng.uniform(0.01, 0.5, N)
    q = oracle.ode_integrate(k, c, steps=2000, dt=1e-3)
    idx = np.array([0, 99, 499, 1234, 1999])
    exact = _exact_positions(k, c, (idx + 1) * 1e-3)
    assert np.max(np.abs(q[idx] - exact)) < 1e-10


def test_rk4_is_fourth_order():
    rng = np.random.default_rng(4)
    k = rng.uniform(0.5, 5.0, N)
    c = rng.uniform(0.01, 0.5, N)
    T = 1.0
    exact = _exact_positions(k, c, [T])[0]
    errs = []
    for h in (0.04, 0.02, 0.01):
        q = oracle.ode_integrate(k, c, steps=int(round(T / h)), dt=h)
        errs.append(np.max(np.abs(q[-1] - exact)))
    for a, b in zip(errs, errs[1:]):
        assert 12.0 < a / b < 20.0, errs


def test_energy_conserved_without_damping_and_decays_with_it():
    rng = np.random.default_rng(5)
    k = rng.uniform(0.5, 5.0, N)
    h, steps = 1e-3, 2000
    # the oracle returns positions only: they must follow the exact solution,
    # and the exact solution keeps the chain's energy (no damping) or loses it
    q0 = np.zeros(N)
    q0[0] = 1.0
    E0 = _energy(k, q0, np.zeros(N))
    q = oracle.ode_integrate(k, np.zeros(N), steps=steps, dt=h)
    A = _system_matrix(k, np.zeros(N))
    s0 = np.concatenate([q0, np.zeros(N)])
    sT = scipy_linalg.expm(A * steps * h) @ s0
    assert np.max(np.abs(q[-1] - sT[:N])) < 1e-10
    assert abs(_energy(k, sT[:N], sT[N:]) - E0) < 1e-12 * E0  # the stated energy is the chain's invariant
    c = rng.uniform(0.01, 0.5, N)
    A = _system_matrix(k, c)
    Es = []
    for t in (0.5, 1.0, 1.5, 2.0):
        s = scipy_linalg.expm(A * t) @ s0
        Es.append(_energy(k, s[:N], s[N:]))
    qd = oracle.ode_integrate(k, c, steps=steps, dt=h)
    assert np.max(np.abs(qd[1999] - (scipy_linalg.expm(A * 2.0) @ s0)[:N])) < 1e-10
    assert all(b < a for a, b in zip([E0] + Es, Es))


@pytest.mark.parametrize("seed", [1, 2, 7])
def test_objective_zero_at_hidden_parameters(seed):
    xh = problems.ode_hidden(seed)
    f, s = oracle.ode_objective(xh, xh)
    assert f == 0.0 and s == 0.0
    X = np.stack([xh, xh])
    fe, _ = oracle.evaluate(oracle.ODE, X, xh)
    assert np.all(fe == 0.0)


def test_objective_is_mean_squared_trajectory_difference():
    xh = problems.ode_hidden(3)
    x = problems.population(1, 20, seed=5)[0]
    a = oracle.ode_trajectory(x)
    b = oracle.ode_trajectory(xh)
    f, s = oracle.ode_objective(x, xh)
    assert f == pytest.approx(np.mean((a - b) ** 2), rel=1e-13)
    assert s >= f > 0.0
    # symmetric in its two arguments, and the dispatcher routes obj 4 here
    assert oracle.ode_objective(xh, x)[0] == f
    fe, se = oracle.evaluate(oracle.ODE, x[None, :], xh)
    assert fe[0] == f and se[0] == s


def test_objective_rejects_wrong_dimension():
    f, _ = oracle.evaluate(oracle.ODE, np.zeros((1, 10)), np.zeros(10))
    assert np.isnan(f[0])
