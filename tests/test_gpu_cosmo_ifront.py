"""The cosmological I-front of Sec. 4.6 ("Cosmological Radiative Ionization") on the GPU.

A 5e48 s^-1 source of 13.6 eV photons ionises uniform hydrogen held at 1e4 K while a
matter-only universe expands; the gas's proper density falls as a^-3, so the Stromgren radius
grows and the front lags behind it.  The library steps the comoving equations: the reaction
terms see proper densities (1/a^3), diffusion a 1/a^2 (reading of the comoving factors), and
with m = 0 (monochromatic radiation) there is no (adot / a) E term.  The run goes from z_i to
z = 0 in intervals of the scale factor, each with (a, adot) at its middle and adaptive implicit
steps inside it (Sec. 3.2.3), through rhi_advance.  The radius of the ionised volume
(x_HII >= 1/2, the corner octant mirrored) follows eq. SG-solution (with eqs. SG-tau and SG-F,
pinned on the CPU against their defining integral) to within 10% at 32^3 cells.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import closure as cl, timestep as ts
from paper_0901_1110_gb300 import inputs

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


@pytest.mark.timeout(900)
@pytest.mark.parametrize("q0,z_i", [(0.5, 4.0), (0.05, 4.0)])
def test_cosmological_ifront_follows_the_analytic_solution(rhi, q0, z_i):
    w = inputs.config_sg(32, q0=q0, z_i=z_i)
    m = w.meta
    a_i, H0, om = m["a_i"], m["H0"], m["omega_m"]
    aB = cl.closure_terms(np.array([1e4]))["alpha_HII_B"][0]
    lam = aB * m["nH_i"] / (H0 * (1.0 + z_i))
    r_Si = (3.0 * m["ndot"] / (4.0 * np.pi * aB * m["nH_i"] ** 2)) ** (1.0 / 3.0)   # proper
    s = rhi.solver_for_workload(w, isothermal=1, m_grey=0, dt_norm=2, dt_tau_tol=0.01,
                                precond=rhi.RHI_PRECOND_MG_FP32, mg_levels=5,
                                limiter_jacobian=2)
    # cosmic time between scale factors from da/dt of the matter-only model
    t_of = lambda a0, a1: integrate.quad(lambda a: 1.0 / inputs.matter_only_adot(a, H0, om),
                                         a0, a1, epsrel=1e-12)[0]
    checks = [1.25, 5.0 / 3.0, 2.5, 10.0 / 3.0, 5.0]            # a / a_i: z = 3, 2, 1, 0.5, 0
    edges = np.unique(np.concatenate([np.geomspace(1.0, 1.0 + z_i, 49), checks]))
    dt, steps, rows = None, 0, []
    for lo, hi in zip(edges[:-1], edges[1:]):
        a_lo, a_hi = lo * a_i, hi * a_i
        a_mid = np.sqrt(a_lo * a_hi)
        span = t_of(a_lo, a_hi)
        adot = float(inputs.matter_only_adot(a_mid, H0, om))
        if dt is None:
            dt = 1e-3 * span
        _, n = s.advance(span, min(dt, span), dt_min=1e-8 * span, a=float(a_mid), adot=adot,
                         newton_tol=1e-7, lin_tol=1e-8)
        steps += n
        dt = max(s.stats()["dt_next"], 1e-8 * span)
        if any(abs(hi - c) < 1e-12 for c in checks):
            st = s.get_state()
            x_HII = 1.0 - np.asarray(st["n"][0]) / w.nH.ravel()
            R = ts.ifront_radius(x_HII, w.dx)          # comoving, a = 1 today
            r = a_i * R / r_Si                         # comoving in units of the initial r_S
            ra = ts.sg_ifront(hi, lam, q0, z_i)[0]
            rows.append((hi, (1.0 + z_i) / hi - 1.0, r, ra, steps))
    print(f"q0 = {q0}, z_i = {z_i}, lambda = {lam:.3f}: (a/a_i, z, r_I/r_S,i, analytic, steps) "
          + str([tuple(round(v, 3) for v in row) for row in rows]))
    for _, _, r, ra, _ in rows:
        assert abs(r / ra - 1.0) < 0.10, rows
    assert steps < 20000
