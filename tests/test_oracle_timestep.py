"""Pins of the adaptive time-step oracle (Sec. 3.2.3): the error estimate of
eq. time_error_estimator is second order in dt (backward Euler against the explicit
predictor), agrees with a cell-by-cell brute-force evaluation, and the I-front helpers
reproduce their closed forms."""
import math

import numpy as np
import pytest

from conftest import oracle_problem
from oracle import closure as cl, model as md, timestep as ts
from paper_0901_1110_gb300 import inputs

KPC = inputs.KPC


def _relaxing_box():
    """A 3^3 hydrogen box with no source, out of ionisation and thermal equilibrium and with a
    decaying radiation field: every component changes smoothly."""
    w = inputs.uniform_h(3, box=30 * KPC, x0=0.3, T0=2e4, E0=1e-17, ndot=0.0)
    w.theta = 1.0
    return w, oracle_problem(w, u_E=1e-17)


def test_error_estimate_is_second_order():
    """U^{n+1} (backward Euler) and U^pred (explicit Euler) both carry O(dt) error, and their
    difference is O(dt^2): halving dt quarters eps_loc.  A first-order difference (a predictor
    with the wrong sign of L, for instance) would only halve it."""
    w, p = _relaxing_box()
    st = w.state()
    eps = []
    for dt in (4e8, 2e8, 1e8):
        _, _, e, _ = ts.step_with_estimate(p, st, dt, 1.0, 0.0, 1e-13, np.inf, 0.01)
        eps.append(e)
    r1, r2 = eps[0] / eps[1], eps[1] / eps[2]
    assert 3.6 < r2 < 4.4, eps
    assert abs(r1 - 4.0) > abs(r2 - 4.0) - 0.05, eps          # tends to 4 as dt -> 0
    for pn in (1.0, 2.0):
        e = [ts.step_with_estimate(p, st, dt, 1.0, 0.0, 1e-13, pn, 0.01)[2]
             for dt in (2e8, 1e8)]
        assert 3.6 < e[0] / e[1] < 4.4, (pn, e)


def test_error_estimate_matches_brute_force():
    rng = np.random.default_rng(3)
    w = inputs.lognormal_hhe((2, 3, 2), nsrc=1)
    p = oracle_problem(w, u_e=2e12, u_n=1e-3, u_E=1e-17)
    Ua = rng.standard_normal((p.nv, p.N)) * p.scales()[:, None] * 3
    Ub = Ua * (1 + 0.1 * rng.standard_normal((p.nv, p.N)))
    u = [p.u_e] + [p.u_n] * p.ns + [p.u_E]
    for pn in (1.0, 2.0, 3.0, np.inf):
        acc, mx = 0.0, 0.0
        for v in range(p.nv):
            for c in range(p.N):
                a, b = Ua[v, c] / u[v], Ub[v, c] / u[v]
                q = abs(a - b) / (math.sqrt(abs(a * b)) + 1.0)
                mx = max(mx, q)
                if not np.isinf(pn):
                    acc += q ** pn
        want = mx if np.isinf(pn) else (acc / (p.N * p.nv)) ** (1.0 / pn)
        assert abs(ts.time_error_estimate(p, Ua, Ub, pn) / want - 1) < 1e-13
    assert ts.time_error_estimate(p, Ua, Ua, 2.0) == 0.0
    assert ts.next_time_step(3e12, 0.02, 0.01) == pytest.approx(1.5e12)


def test_ifront_helpers():
    """Eq. Ifront_solution at t = t_rec is (1 - 1/e)^(1/3) r_S and tends to r_S; the mirrored
    ionised-volume radius of a discretised ball of radius R is R to within a cell."""
    r = ts.ifront_analytic([3.86e15, 1e18], 5.4, 3.86e15)
    assert r[0] == pytest.approx(5.4 * (1 - math.exp(-1)) ** (1 / 3), rel=1e-14)
    assert r[1] == pytest.approx(5.4, rel=1e-12)
    n, dx, R = 40, 0.25, 7.3
    c = (np.arange(n) + 0.5) * dx
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    x = np.where(np.sqrt(X ** 2 + Y ** 2 + Z ** 2) <= R, 0.9, 0.1)
    assert abs(ts.ifront_radius(x, dx) - R) < dx
    # the case-B coefficient of the closure gives the printed Stromgren radius
    aB = cl.rate_formulas(np.array([1e4]))[0, 0]
    rS = (3 * 5e48 / (4 * np.pi * aB * 1e-3 ** 2)) ** (1 / 3) / KPC
    assert rS == pytest.approx(5.4, rel=0.01)


@pytest.mark.parametrize("q0,z_i", [(0.5, 4.0), (0.05, 4.0), (0.5, 10.0), (0.05, 10.0)])
def test_sg_tau_closed_form_is_its_integral(q0, z_i):
    """Eq. SG-tau with eq. SG-F is the closed form of the recombination depth
    lambda int_1^a a'^-3 g(a') da' with H0 (1 + z_i) dt = g da (matter and curvature only):
    quadrature of that definition agrees for the four parameter pairs of the paper."""
    from scipy import integrate
    lam = 2.246
    for a in (1.0, 1.3, 2.0, 5.0, 11.0):
        q, _ = integrate.quad(lambda x: lam * x ** -3 * ts.sg_g(x, q0, z_i), 1.0, a,
                              epsabs=0.0, epsrel=1e-13)
        assert ts.sg_tau(a, lam, q0, z_i) == pytest.approx(q, rel=1e-11, abs=1e-14)


def test_sg_ifront_limits():
    """Eq. SG-solution: at early times photon counting, r_I^3 = r_S,i^3 lam g(1) (a - 1)
    (no recombinations yet); for fast recombination (lam -> inf) the comoving Stromgren radius
    of the diluted gas, r_S,i a (r_S proper grows as a^2 with n ~ a^-3); and in between the
    front lags that Stromgren radius."""
    q0, z_i = 0.5, 4.0
    lam = 2.246
    a = 1.0 + 1e-5
    r = ts.sg_ifront(a, lam, q0, z_i)[0]
    assert r ** 3 == pytest.approx(lam * ts.sg_g(1.0, q0, z_i) * 1e-5, rel=1e-4)
    for a in (1.5, 3.0):
        assert ts.sg_ifront(a, 1e5, q0, z_i)[0] == pytest.approx(a, rel=1e-3)
    r = ts.sg_ifront([1.25, 2.5, 5.0], lam, q0, z_i)
    assert np.all(np.diff(r) > 0) and np.all(r < np.array([1.25, 2.5, 5.0]))
