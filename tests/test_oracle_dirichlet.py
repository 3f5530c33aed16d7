"""Pins of the oracle's Dirichlet boundaries (the boundary value sits on the face, half a cell
from the cell centre): the Newton matrix against central differences with boundary faces, and
the steady diffusion profile between two Dirichlet values, which the scheme reproduces as the
exact straight line."""
import numpy as np
import pytest

from conftest import oracle_problem
from oracle import closure as cl, model as md, solve as sv
from paper_0901_1110_gb300 import inputs
from test_oracle_lte import _fd

KPC = inputs.KPC


@pytest.mark.parametrize("ljac", ["lagged", "E", "exact"])
@pytest.mark.parametrize("model", ["ionization", "lte"])
def test_jacobian_with_dirichlet_faces(ljac, model):
    rng = np.random.default_rng(7)
    bc = ("dirichlet", "dirichlet", "zero_flux", "zero_flux", "dirichlet", "periodic")
    bcz = ("dirichlet", "dirichlet", "zero_flux", "zero_flux", "periodic", "periodic")
    if model == "lte":
        w = inputs.lte_uniform(7e7, n=3, box=3e11, E_perturb=0.3, dt=1e-9, bc=bcz)
        vals = (3e12, 2e11, 0, 0, 0, 0)
    else:
        w = inputs.uniform_h(3, shape=(2, 3, 3), box=60 * KPC, dt=3e13, bc=bcz)
        w.E = 1e-17 * np.exp(rng.uniform(-3, 3, w.E.shape))
        w.n = w.n * rng.uniform(0.001, 1.0, w.n.shape)
        vals = (5e-16, 1e-18, 0, 0, 0, 0)
    p = oracle_problem(w, limiter_jacobian=ljac, theta=0.8, bc_value=vals,
                       **({"u_E": 1e-17} if model != "lte" else {}))
    st = w.state()
    U = md.state_to_U(p, st)
    eh = st["e"]
    U[0] = 0.1 * eh * rng.standard_normal(p.N)
    g = md.build_g(p, md.state_to_U(p, st), eh, w.dt, 1.0, 0.0)
    if ljac == "lagged":
        lt = md.local_terms(p, U[0], U[1:1 + p.ns], U[1 + p.ns], eh, p.nH, p.src, 1.0, 0.0)
        W = md.face_weights(p, U[1 + p.ns], lt["kappa"], 1.0)
        from test_oracle_model import _fd_jacobian
        Jfd = _fd_jacobian(p, U, g, eh, w.dt, 1.0, 0.0, None, W)
        tol = 1e-6
    elif ljac == "E":
        lt = md.local_terms(p, U[0], U[1:1 + p.ns], U[1 + p.ns], eh, p.nH, p.src, 1.0, 0.0)
        from test_oracle_model import _fd_jacobian
        Jfd = _fd_jacobian(p, U, g, eh, w.dt, 1.0, 0.0, None, kap_faces=lt["kappa"])
        tol = 3e-5
    else:
        Jfd = _fd(p, U, g, eh, w.dt)
        tol = 3e-5
    J = md.full_jacobian(p, U, eh, w.dt, 1.0, 0.0).toarray()
    scale = np.abs(Jfd).max(axis=1, keepdims=True)
    assert np.max(np.abs(J - Jfd) / scale) < tol


def test_steady_diffusion_between_dirichlet_values_is_a_straight_line():
    """LTE medium with kappa L << 1 and no emission, limiter off (D = c / (3 kappa)):
    backward-Euler steps of 1000 times the slowest diffusion time (pi^2 D / L^2 ~ 1e17 / s)
    reach the steady profile, which the half-cell boundary faces make exactly
    E_L + (E_R - E_L) x / L at the cell centres (up to the absorption, 3 kappa^2 L^2 ~ 3e-12
    of the profile)."""
    n, L = 16, 1.0
    bc = ("dirichlet", "dirichlet", "zero_flux", "zero_flux", "zero_flux", "zero_flux")
    w = inputs.lte_uniform(1.0, n=n, rho=1.0, E0=0.5, kappa=1e-6, box=L, dt=1e-6, bc=bc)
    w.kappa_planck = 0.0
    p = oracle_problem(w, limiter=False, bc_value=(2.0, 1.0, 0, 0, 0, 0), u_e=1.0, u_E=1.0)
    new = w.state()
    for _ in range(4):
        new, info = sv.implicit_step(p, new, 1e-14, 1.0, 0.0, 1e-10, linear="direct")
        assert info["converged"]
    x = (np.arange(n) + 0.5) * (L / n)
    want = 2.0 + (1.0 - 2.0) * x / L
    E = np.asarray(new["E"]).reshape(n, n, n)
    assert np.abs(E - want[None, None, :]).max() < 1e-9
