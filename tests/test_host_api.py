"""Host-only entry points of the C ABI, run on the CPU (they touch no device): the documented
parameter defaults, the argument checks of rhi_params_default, and the grey constants of eq.
adaptive_spectrum against the oracle's quadrature."""
import math

import numpy as np
import pytest

from oracle import closure as cl


@pytest.fixture(scope="module")
def rhi():
    from paper_0901_1110_gb300 import _build
    _build.build()
    import paper_0901_1110_gb300 as rhi
    rhi.lib()
    return rhi


@pytest.mark.parametrize("ns", [0, 1, 3])
def test_params_default_match_the_header(rhi, ns):
    p = rhi.rhi_params_default(ns)
    expect = dict(n_species=ns, theta=0.51, m_grey=1, isothermal=0, limiter=1,
                  kappa_floor=1e-40, u_e=1.0, u_n=1.0, u_E=1.0, tau=0.99, lam_min=1.0 / 16.0,
                  mlp_gate=1e-3, mlp_ood=6.0, mlp_restart=12, mlp_retry=4, growth_max=1e3,
                  watchdog=3, limiter_jacobian=0, max_newton=50, max_pcg=200,
                  guess=rhi.RHI_GUESS_PREVIOUS, precond=rhi.RHI_PRECOND_MG_FP64, mg_levels=6,
                  mg_pre=2, mg_post=2, mg_coarse_sweeps=16, mg_omega=0.9, vcycle_graph=1,
                  krylov_graph=1, mg_matrix=1, krylov_restart=-1.0, predict_final=1, dt_norm=0, dt_tau_tol=0.01, mu=0.6,
                  model=rhi.RHI_MODEL_LTE if ns == 0 else rhi.RHI_MODEL_IONIZATION)
    for k, v in expect.items():
        assert getattr(p, k) == v, k
    # 13.6 eV monochromatic grey constants: HI absorbs at 6.3e-18 cm^2, helium not at all
    assert math.isclose(p.photon_energy, 13.6 * cl.EV, rel_tol=1e-12)
    if ns >= 1:
        assert math.isclose(p.sk[0], 6.3e-18, rel_tol=1e-12)
    assert p.sk[1] == 0.0 and p.sk[2] == 0.0


@pytest.mark.parametrize("ns", [-1, 2, 4])
def test_params_default_rejects_species_counts(rhi, ns):
    with pytest.raises(rhi.RhiError) as e:
        rhi.rhi_params_default(ns)
    assert e.value.code == rhi.RHI_ERR_ARG


@pytest.mark.parametrize("spec,par,ns", [("blackbody", 1e5, 3), ("blackbody", 3e4, 1),
                                         ("powerlaw", -1.7, 3), ("powerlaw", -3.0, 3),
                                         ("mono", 13.6, 1), ("mono", 30.0, 3)])
def test_grey_constants_match_oracle_quadrature(rhi, spec, par, ns):
    """Library closed forms (Bose series, E1) against the oracle's adaptive quadrature of eq.
    adaptive_spectrum; absorbers beyond n_species are 0."""
    code = {"blackbody": rhi.RHI_SPECTRUM_BLACKBODY, "powerlaw": rhi.RHI_SPECTRUM_POWERLAW,
            "mono": rhi.RHI_SPECTRUM_MONO}[spec]
    param = par * cl.EV if spec == "mono" else par
    a = rhi.rhi_grey_constants(code, param, ns)
    b = cl.grey_constants(spec, param, ns)
    for k in ("sk", "pgam", "ph"):
        np.testing.assert_allclose(a[k], b[k], rtol=1e-11, atol=0)
        assert np.all(np.asarray(a[k])[ns:] == 0.0)
    assert abs(a["eps"] / b["eps"] - 1) < 1e-12


# ---- argument checks of rhi_create: every one returns before any device call

def _create(rhi, shape=(4, 5, 6), dx=1e21, bc=None, bc_value=(0.0,) * 6, **tweak):
    p = rhi.rhi_params_default(3)
    p.y_he = 0.0789
    for k, v in tweak.items():
        setattr(p, k, v)
    kinds = bc if bc is not None else (rhi.RHI_BC_ZERO_FLUX,) * 6
    return rhi.Solver(*shape, dx, p, bc=kinds, bc_value=bc_value)


@pytest.mark.parametrize("shape,dx", [((0, 4, 4), 1e21), ((4, -1, 4), 1e21), ((4, 4, 4), 0.0),
                                      ((4, 4, 4), float("nan")), ((2048, 2048, 1024), 1e21)])
def test_create_rejects_bad_grids(rhi, shape, dx):
    with pytest.raises(rhi.RhiError) as e:
        _create(rhi, shape=shape, dx=dx)
    assert e.value.code == rhi.RHI_ERR_ARG


def test_create_rejects_bad_boundaries(rhi):
    Z, P, D = rhi.RHI_BC_ZERO_FLUX, rhi.RHI_BC_PERIODIC, rhi.RHI_BC_DIRICHLET
    for bc, val in (((P, Z, Z, Z, Z, Z), (0.0,) * 6),            # unpaired periodic
                    ((Z, Z, 7, Z, Z, Z), (0.0,) * 6),            # unknown kind
                    ((D, Z, Z, Z, Z, Z), (0.0,) * 6),            # Dirichlet value must be > 0
                    ((Z, D, Z, Z, Z, Z), (0.0, float("inf"), 0, 0, 0, 0))):
        with pytest.raises(rhi.RhiError) as e:
            _create(rhi, bc=bc, bc_value=val)
        assert e.value.code == rhi.RHI_ERR_ARG, bc


@pytest.mark.parametrize("tweak", [
    dict(n_species=2), dict(theta=0.0), dict(theta=1.5), dict(u_E=0.0), dict(tau=1.0),
    dict(lam_min=0.0), dict(growth_max=0.5), dict(watchdog=-1), dict(max_pcg=0),
    dict(guess=9), dict(mlp_gate=-1.0), dict(mlp_retry=-1), dict(precond=7), dict(mg_levels=0),
    dict(mg_pre=0), dict(mg_coarse_sweeps=0), dict(limiter_jacobian=3), dict(mg_omega=1.5),
    dict(vcycle_graph=2), dict(krylov_graph=2), dict(mg_matrix=2), dict(krylov_restart=1.0),
    dict(krylov_restart=float("nan")), dict(predict_final=2), dict(dt_norm=-2), dict(dt_tau_tol=0.0), dict(y_he=-0.1),
    dict(model=1)])                                   # the LTE model needs n_species = 0
def test_create_rejects_out_of_range_parameters(rhi, tweak):
    with pytest.raises(rhi.RhiError) as e:
        _create(rhi, **tweak)
    assert e.value.code == rhi.RHI_ERR_ARG


def test_null_handles_and_status_strings(rhi):
    lib = rhi.lib()
    assert lib.rhi_set_state(None, None, None, None, None, None, 0) == rhi.RHI_ERR_ARG
    assert lib.rhi_implicit_step(None, 1.0, 1.0, 0.0, 1e-8, 1e-10) == rhi.RHI_ERR_ARG
    assert lib.rhi_get_state(None, None, None, None, 0) == rhi.RHI_ERR_ARG
    assert lib.rhi_get_stats(None, None) == rhi.RHI_ERR_ARG
    assert lib.rhi_last_error(None) == b"null handle"
    texts = {lib.rhi_status_string(c) for c in (rhi.RHI_OK, rhi.RHI_ERR_ARG, rhi.RHI_ERR_CUDA,
                                                rhi.RHI_ERR_NONCONVERGED,
                                                rhi.RHI_ERR_NONPHYSICAL, rhi.RHI_ERR_STATE)}
    assert len(texts) == 6 and lib.rhi_status_string(99) == b"unknown status"
