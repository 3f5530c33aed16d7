"""The LTE coupling model (eq. LTE_coupling) on the GPU: implicit steps vs the FP64 oracle, and
the matter-radiation equilibration test of Sec. 4.2 (Turner & Stone) with its closed-system
equilibrium and total-energy conservation."""
import numpy as np
import pytest
from scipy.optimize import brentq

from conftest import oracle_problem
from oracle import closure as cl, solve as sv
from paper_0901_1110_gb300 import inputs
from parity import TIGHT_NEWTON_TOL, field_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rhi():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_0901_1110_gb300 import _build
    _build.build()
    import paper_0901_1110_gb300 as rhi
    rhi.lib()
    return rhi


@pytest.mark.parametrize("ljac,theta", [(0, 1.0), (2, 1.0), (2, 0.7)])
def test_lte_steps_match_oracle(rhi, ljac, theta):
    """Gas near the radiation temperature in a periodic 6^3 box with a perturbed field, so
    that emission, absorption and flux-limited diffusion all act."""
    w = inputs.lte_uniform(7e7, n=6, box=3e11, E_perturb=0.3, dt=3e-10, seed=2)
    w.nH = w.nH * np.exp(np.random.default_rng(3).uniform(-0.4, 0.4, w.nH.shape))
    w.theta = theta
    s = rhi.solver_for_workload(w, limiter_jacobian=ljac, precond=rhi.RHI_PRECOND_MG_FP32,
                                mg_levels=2)
    p = oracle_problem(w)
    ref = w.state()
    for _ in range(3):
        s.step(w.dt, newton_tol=TIGHT_NEWTON_TOL, lin_tol=1e-12)
        ref, info = sv.implicit_step(p, ref, w.dt, 1.0, 0.0, TIGHT_NEWTON_TOL, linear="direct")
        assert info["converged"]
        err = field_errors(s.get_state(), ref, w.nH, scales=(w.u_e, w.u_n, w.u_E))
        assert max(err.values()) <= 1e-10, err


def _equilibrium(rho, mu, e_vol0, E0):
    Etot = e_vol0 + E0
    cv = rho * cl.K_BOLTZ / ((cl.GAMMA - 1.0) * mu * cl.M_H)
    T = brentq(lambda T: cv * T + cl.A_RAD * T ** 4 - Etot, 1.0, 1e10, xtol=1e-14, rtol=1e-15)
    return cv * T


@pytest.mark.parametrize("e_vol0", [1e10, 1e2])
def test_turner_stone_on_gpu(rhi, e_vol0):
    """4^3 periodic box, kappa = 4e-8 cm^-1, rho = 1e-7 g cm^-3, mu = 0.6, E = 1e12 erg cm^-3:
    the gas energy reaches the equilibrium of the closed system, and the relative drift of
    the total energy (the paper's conservation measure) stays below 1e-11."""
    w = inputs.lte_uniform(e_vol0, n=4)
    s = rhi.solver_for_workload(w, u_e=1e17, precond=rhi.RHI_PRECOND_MG_FP32, mg_levels=2,
                                limiter_jacobian=2)
    rho = 1e-7
    st = w.state()
    E_tot0 = (rho * st["e"] + st["E"]).sum()
    t, dt = 0.0, 1e-12
    while t < 2e-6:
        s.step(dt, newton_tol=1e-10, lin_tol=1e-9)
        t += dt
        dt = min(2 * dt, 2e-7)
    g = s.get_state()
    e_eq = _equilibrium(rho, 0.6, e_vol0, 1e12)
    assert np.allclose(rho * np.asarray(g["e"]), e_eq, rtol=1e-6)
    drift = np.abs(rho * np.asarray(g["e"]) + np.asarray(g["E"]) - (rho * st["e"] + st["E"])).sum() / E_tot0
    print(f"e_vol0 = {e_vol0:g}: relative total-energy drift {drift:.2e}")
    assert drift < 1e-11


def test_lte_argument_errors(rhi):
    p = rhi.rhi_params_default(0)
    assert p.model == rhi.RHI_MODEL_LTE
    p.kappa_total = p.kappa_planck = 1e-6
    p.guess = rhi.RHI_GUESS_LEARNED
    with pytest.raises(rhi.RhiError):
        rhi.Solver(2, 2, 2, 1.0, p)
    p.guess = rhi.RHI_GUESS_PREVIOUS
    p.model = rhi.RHI_MODEL_IONIZATION
    with pytest.raises(rhi.RhiError):
        rhi.Solver(2, 2, 2, 1.0, p)
