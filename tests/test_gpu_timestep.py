"""Adaptive time stepping (Sec. 3.2.3) on the GPU: the error estimate against the explicit
predictor and the next step size vs the oracle, and the HII-region test of Sec. 4.5 run with
adaptive steps against the analytic I-front radius (eq. Ifront_solution)."""
import numpy as np
import pytest

from conftest import oracle_problem
from oracle import timestep as ts
from paper_0901_1110_gb300 import inputs

pytestmark = pytest.mark.gpu
KPC = inputs.KPC
MYR = 3.15576e13


@pytest.fixture(scope="module")
def rhi():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_0901_1110_gb300 import _build
    _build.build()
    import paper_0901_1110_gb300 as rhi
    rhi.lib()
    return rhi


@pytest.mark.parametrize("p_norm", [2, -1])
@pytest.mark.parametrize("guess", ["prev", "predictor"])
def test_error_estimate_and_next_step_match_oracle(rhi, p_norm, guess):
    w = inputs.lognormal_hhe((9, 10, 11), box=150 * KPC, nsrc=2, dt=2e12, seed=4)
    w.theta = 1.0
    w.u_E = 1e-18
    code = rhi.RHI_GUESS_PREVIOUS if guess == "prev" else rhi.RHI_GUESS_PREDICTOR
    s = rhi.solver_for_workload(w, dt_norm=p_norm, dt_tau_tol=0.02, guess=code)
    p = oracle_problem(w)
    st = w.state()
    for _ in range(2):
        s.step(w.dt, newton_tol=1e-12, lin_tol=1e-12)
        g = s.stats()
        st, _, eps, dtn = ts.step_with_estimate(p, st, w.dt, 1.0, 0.0, 1e-13,
                                                np.inf if p_norm < 0 else float(p_norm), 0.02)
        assert abs(g["eps_loc"] / eps - 1) < 1e-7, (g["eps_loc"], eps)
        assert abs(g["dt_next"] / dtn - 1) < 1e-7


def test_hii_region_front_follows_the_analytic_solution(rhi):
    """Sec. 4.5: 6.6 kpc box, n_H = 1e-3, T = 1e4 K held fixed, x_HII = 0.0012, E = 1e-20,
    a 5e48 s^-1 13.6 eV source in the corner cell (the octant's eighth of it), adaptive steps
    with p = 2 and tau_tol = 0.01.  The mirrored ionised-volume radius follows
    r_S (1 - exp(-t / t_rec))^(1/3) to within 8% from 0.5 t_rec to 4 t_rec."""
    n = 32
    w = inputs.uniform_h(n, box=6.6 * KPC, nH=1e-3, T0=1e4, x0=0.0012, E0=1e-20,
                         ndot=5e48 / 8, source="corner")
    w.theta = 1.0
    s = rhi.solver_for_workload(w, isothermal=1, dt_norm=2, dt_tau_tol=0.01, u_E=1e-17,
                                precond=rhi.RHI_PRECOND_MG_FP32, mg_levels=4,
                                limiter_jacobian=2)
    aB = 2.59e-13
    r_S = (3 * 5e48 / (4 * np.pi * aB * 1e-6)) ** (1 / 3)
    t_rec = 1.0 / (aB * 1e-3)
    t, dt, total_steps = 0.0, 1e10, 0
    rows = []
    for frac in (0.5, 1.0, 2.0, 4.0):
        t_goal = frac * t_rec
        t_now, steps = s.advance(t_goal - t, dt, dt_min=1e6, newton_tol=1e-7, lin_tol=1e-8)
        t += t_now
        total_steps += steps
        dt = max(s.stats()["dt_next"], 1e6)
        st = s.get_state()
        x_HII = 1.0 - np.asarray(st["n"][0]) / w.nH.ravel()
        r = ts.ifront_radius(x_HII, w.dx)
        ra = ts.ifront_analytic(t, r_S, t_rec)
        rows.append((t / t_rec, r / KPC, ra / KPC, total_steps))
    print("t/t_rec, r_I (kpc), analytic (kpc), steps:", [tuple(round(v, 3) for v in r) for r in rows])
    for tf, r, ra, _ in rows:
        assert abs(r / ra - 1) < 0.08, rows
    assert total_steps < 5000


def test_advance_argument_errors(rhi):
    w = inputs.uniform_h(4, dt=1e12)
    s = rhi.solver_for_workload(w)                    # dt_norm = 0
    with pytest.raises(rhi.RhiError):
        s.advance(1e13, 1e12)
    s2 = rhi.solver_for_workload(w, dt_norm=2)
    with pytest.raises(rhi.RhiError):
        s2.advance(1e13, -1.0)
    t, n = s2.advance(3e12, 1e12, dt_max=1e12)
    assert n >= 3 and abs(t / 3e12 - 1) < 1e-12          # no step above dt_max
    t, n = s2.advance(3e12, 1e12, dt_min=1e12, dt_max=1e12)
    assert n == 3 and abs(t / 3e12 - 1) < 1e-12          # dt clamped to 1e12 exactly
