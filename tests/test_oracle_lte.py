"""Pins of the oracle's LTE coupling model (eq. LTE_coupling): the Newton matrix against central
differences, and the matter-radiation equilibration of Sec. 4.2 (Turner & Stone): the gas
energy reaches the equilibrium of the closed system, and the total energy is conserved to the
Newton tolerance (the paper's conservation table)."""
import numpy as np
import pytest
from scipy.optimize import brentq

from conftest import oracle_problem
from oracle import closure as cl, model as md, solve as sv
from paper_0901_1110_gb300 import inputs


def _fd(p, U, g, eh, dt):
    u = p.scales()
    J = np.zeros((p.nv * p.N, p.nv * p.N))
    for v in range(p.nv):
        for c in range(p.N):
            h = 1e-6 * max(abs(U[v, c]), 1e-3 * u[v])
            Up = U.copy(); Up[v, c] += h
            Um = U.copy(); Um[v, c] -= h
            fp = md.residual(p, Up, g, eh, dt, 1.0, 0.0) / u[:, None]
            fm = md.residual(p, Um, g, eh, dt, 1.0, 0.0) / u[:, None]
            J[:, v * p.N + c] = ((fp - fm) / (2 * h) * u[v]).ravel()
    return J


@pytest.mark.parametrize("ljac", ["lagged", "exact"])
def test_lte_jacobian_matches_central_differences(ljac):
    # gas near the radiation temperature (3.4e6 K), so that emission and absorption both count
    w = inputs.lte_uniform(7e7, n=2, box=3e11, E_perturb=0.3, dt=1e-9)
    w.nH = w.nH * np.exp(np.random.default_rng(1).uniform(-0.5, 0.5, w.nH.shape))
    p = oracle_problem(w, limiter_jacobian=ljac, theta=0.7)
    rng = np.random.default_rng(2)
    st = w.state()
    U = md.state_to_U(p, st)
    eh = st["e"]
    U[0] = 0.2 * eh * rng.standard_normal(p.N)
    U[1] *= 1 + 0.3 * rng.standard_normal(p.N)
    g = md.build_g(p, md.state_to_U(p, st), eh, w.dt, 1.0, 0.0)
    J = md.full_jacobian(p, U, eh, w.dt, 1.0, 0.0).toarray()
    Jfd = _fd(p, U, g, eh, w.dt)
    scale = np.abs(Jfd).max(axis=1, keepdims=True)
    if ljac == "exact":
        assert np.max(np.abs(J - Jfd) / scale) < 3e-5
    else:     # D lagged: only the E-E block differs, by the limiter's E dependence
        assert np.max(np.abs((J - Jfd)[:p.N]) / scale[:p.N]) < 1e-6


def _equilibrium(rho, mu, e_vol0, E0):
    """The closed system's equilibrium: rho e + E conserved and c kappa E = 4 kappa sigma T^4
    (one opacity), i.e. E = a_r T^4 with e = k_B T / ((gamma - 1) mu m_H)."""
    Etot = e_vol0 + E0
    cv = rho * cl.K_BOLTZ / ((cl.GAMMA - 1.0) * mu * cl.M_H)          # rho e = cv T
    T = brentq(lambda T: cv * T + cl.A_RAD * T ** 4 - Etot, 1.0, 1e10, xtol=1e-14, rtol=1e-15)
    return cv * T, cl.A_RAD * T ** 4


@pytest.mark.parametrize("e_vol0", [1e10, 1e2])
def test_turner_stone_equilibration_and_conservation(e_vol0):
    w = inputs.lte_uniform(e_vol0, n=2, E_perturb=0.0)
    p = oracle_problem(w, u_e=1e10 / 1e-7)
    st = w.state()
    rho = 1e-7
    Etot0 = rho * st["e"] + st["E"]
    # the gas relaxes on rho c_v / (16 kappa sigma T^3) ~ 1.4e-8 s; backward Euler steps of
    # up to 2e-7 s reach the discrete equilibrium, which is the true one (L(U) = 0)
    t, dt = 0.0, 1e-12
    while t < 2e-6:
        st, info = sv.implicit_step(p, st, dt, 1.0, 0.0, 1e-12, linear="direct")
        assert info["converged"]
        t += dt
        dt = min(2 * dt, 2e-7)
    e_eq, E_eq = _equilibrium(rho, 0.6, e_vol0, 1e12)
    assert np.allclose(rho * st["e"], e_eq, rtol=1e-6), (rho * st["e"][0], e_eq)
    # the paper's closed form e_eq = (3/2) (rho k_B / (0.6 m_H)) (E / a_r)^(1/4) holds at the
    # initial E; the radiation gives or takes at most e_vol0 + e_eq, which moves T^4 by that
    # fraction of E and e_eq by a quarter of it
    e_ts = 1.5 * rho * cl.K_BOLTZ / (0.6 * cl.M_H) * (1e12 / cl.A_RAD) ** 0.25
    assert abs(e_eq / e_ts - 1) < 0.26 * (e_vol0 + e_eq) / 1e12 + 1e-9
    drift = np.abs(rho * st["e"] + st["E"] - Etot0).sum() / Etot0.sum()
    assert drift < 1e-10, drift
