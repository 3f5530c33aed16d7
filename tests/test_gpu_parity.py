"""GPU (CUDA path through the C ABI) vs the FP64 oracle on the same seeded inputs."""
import numpy as np
import pytest

from conftest import oracle_problem
from oracle import closure as cl, model as md, solve as sv
from paper_0901_1110_gb300 import inputs
from parity import TIGHT_NEWTON_TOL, field_errors

pytestmark = pytest.mark.gpu
KPC = inputs.KPC

# bound on the per-element error of every field and species fraction (parity.field_errors:
# max |gpu - oracle| / (|oracle| + 1e-12 max|oracle|)) for the FP64 path at tight tolerances
TOL_FP64 = 1e-10


@pytest.fixture(scope="module")
def rhi():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_0901_1110_gb300 import _build
    _build.build()
    import paper_0901_1110_gb300 as rhi
    rhi.lib()
    return rhi


def _field_errors(gpu, ref, w, mask=None):
    return field_errors(gpu, ref, w.nH, w.y_he, mask=mask, scales=(w.u_e, w.u_n, w.u_E))


def _workloads():
    w1 = inputs.uniform_h(6, shape=(9, 10, 11), box=60 * KPC, dt=3e12, nsteps=3, E0=1e-19)
    w1.theta = 1.0
    w1.u_E = 1e-18
    w2 = inputs.lognormal_hhe((18, 20, 24), box=200 * KPC, nsrc=3, dt=5e12, nsteps=3)
    w2.theta = 1.0
    w2.u_E = 1e-18
    w3 = inputs.lognormal_hhe((8, 13, 16), box=150 * KPC, nsrc=2, dt=5e12, nsteps=2,
                              bc=("periodic",) * 6, seed=3)
    w3.theta = 1.0
    w3.u_E = 1e-18
    # theta < 1 keeps E positive only while (1 - theta) c kappa dt < 1: a short step
    w4 = inputs.uniform_h(6, shape=(9, 10, 11), box=60 * KPC, dt=5e9, nsteps=3, E0=1e-19)
    w4.theta = 0.6
    w4.u_E = 1e-18
    return {"uniform_h_ragged": w1, "lognormal_hhe": w2, "lognormal_hhe_periodic": w3,
            "uniform_h_theta06": w4}


WL = _workloads()


def test_grey_constants_match_oracle_quadrature(rhi):
    """Library closed forms vs oracle quadrature of eq. adaptive_spectrum."""
    for spec, par, code in (("blackbody", 1e5, rhi.RHI_SPECTRUM_BLACKBODY),
                            ("powerlaw", -1.7, rhi.RHI_SPECTRUM_POWERLAW),
                            ("mono", 13.6 * cl.EV, rhi.RHI_SPECTRUM_MONO)):
        a = rhi.rhi_grey_constants(code, par, 3)
        b = cl.grey_constants(spec, par, 3)
        for k in ("sk", "pgam", "ph"):
            np.testing.assert_allclose(a[k], b[k], rtol=1e-11, atol=0)
        assert abs(a["eps"] / b["eps"] - 1) < 1e-12


LJAC = {0: "lagged", 1: "E", 2: "exact"}


@pytest.mark.parametrize("ljac", [0, 1, 2])
@pytest.mark.parametrize("name", list(WL))
def test_linear_system_matches_oracle(rhi, name, ljac):
    """Residual f(U^n) (eq. nonlinear_residual), Schur matrix S = D - L M^-1 U and right-hand
    side L M^-1 f_M - f_E (Sec. 3.2.1) of the first Newton system, cell by cell, with D lagged
    (symmetric S), with dD/dE kept, and exact (dD/dE and D's opacity dependence kept: the E
    rows reach the neighbours' species, folded into S by the cell-local elimination)."""
    w = WL[name]
    s = rhi.solver_for_workload(w, limiter_jacobian=ljac)
    lin = s.linearize(w.dt)
    p = oracle_problem(w, limiter_jacobian=LJAC[ljac])
    st = w.state()
    U = md.state_to_U(p, st)
    g = md.build_g(p, U, st["e"], w.dt, 1.0, 0.0)
    f = md.residual(p, U, g, st["e"], w.dt, 1.0, 0.0)
    fs = f / p.scales()[:, None]
    S, rhs, _, _ = sv.schur_system(p, U, f, st["e"], w.dt, 1.0, 0.0)
    for v in range(p.nv):
        scale = max(np.abs(fs[v]).max(), 1e-300)
        assert np.abs(lin["f"][v] - fs[v]).max() <= 1e-12 * scale, v
    # the Schur diagonal and right-hand side subtract L M^-1 U / L M^-1 f_M: cancellation
    np.testing.assert_allclose(lin["diag"], S.diagonal(), rtol=TOL_FP64)
    np.testing.assert_allclose(lin["rhs"], rhs, rtol=TOL_FP64, atol=1e-12 * np.abs(rhs).max())
    # face entries: a cell's coupling to its lower (d = 2 ax) and upper (2 ax + 1) neighbours
    nb, valid = md.neighbor_table(p)
    Sd = S.tocsr()
    dims = (p.nx, p.ny, p.nz)
    for ax in range(3):
        if p.bc[2 * ax] == "periodic" and dims[ax] <= 2:
            continue                      # both faces join the same pair of cells
        for d, key in ((2 * ax, "face"), (2 * ax + 1, "face_hi")):
            want = np.where(valid[d], -np.asarray(Sd[np.arange(p.N), nb[d]]).ravel(), 0.0)
            scale = max(np.abs(want).max(), 1e-300)
            assert np.abs(lin[key][ax] - want).max() <= 1e-11 * scale, (ax, key)


@pytest.mark.parametrize("name", list(WL))
@pytest.mark.parametrize("precond", ["jacobi", "mg64", "mg32"])
def test_steps_match_oracle(rhi, name, precond):
    """Several implicit steps: every field and species fraction within 1e-10 per element of the
    oracle's Newton solution with exact linear solves."""
    w = WL[name]
    code = {"jacobi": rhi.RHI_PRECOND_JACOBI, "mg64": rhi.RHI_PRECOND_MG_FP64,
            "mg32": rhi.RHI_PRECOND_MG_FP32}[precond]
    s = rhi.solver_for_workload(w, precond=code, mg_levels=4)
    p = oracle_problem(w)
    ref = w.state()
    for step in range(w.nsteps):
        s.step(w.dt, 1.0, 0.0, newton_tol=TIGHT_NEWTON_TOL, lin_tol=1e-12)
        ref, stats = sv.implicit_step(p, ref, w.dt, 1.0, 0.0, TIGHT_NEWTON_TOL, linear="direct")
        assert stats["converged"]
        err = _field_errors(s.get_state(), ref, w)
        assert max(err.values()) <= TOL_FP64, (step, err, s.stats())


@pytest.mark.parametrize("ljac", [1, 2])
@pytest.mark.parametrize("name", ["lognormal_hhe", "lognormal_hhe_periodic", "uniform_h_ragged"])
def test_steps_with_dD_dE_match_oracle(rhi, name, ljac):
    """The Newton matrices that keep dD/dE, or are exact (BiCGStab on the non-symmetric Schur
    matrix, preconditioned by the FP32 V-cycle), reach the same solution as the oracle."""
    w = WL[name]
    s = rhi.solver_for_workload(w, precond=rhi.RHI_PRECOND_MG_FP32, mg_levels=4,
                                limiter_jacobian=ljac)
    p = oracle_problem(w)
    ref = w.state()
    for step in range(w.nsteps):
        s.step(w.dt, 1.0, 0.0, newton_tol=TIGHT_NEWTON_TOL, lin_tol=1e-12)
        ref, stats = sv.implicit_step(p, ref, w.dt, 1.0, 0.0, TIGHT_NEWTON_TOL, linear="direct")
        err = _field_errors(s.get_state(), ref, w)
        assert max(err.values()) <= TOL_FP64, (step, err, s.stats())


def test_predictor_guess_reaches_the_same_root(rhi):
    """Eq. explicit_predictor as the Newton initial guess: same solution as U^n."""
    w = WL["lognormal_hhe"]
    a = rhi.solver_for_workload(w, guess=rhi.RHI_GUESS_PREDICTOR)
    a.step(w.dt, newton_tol=TIGHT_NEWTON_TOL, lin_tol=1e-12)
    p = oracle_problem(w)
    ref, _ = sv.implicit_step(p, w.state(), w.dt, 1.0, 0.0, TIGHT_NEWTON_TOL, guess="predictor")
    assert max(_field_errors(a.get_state(), ref, w).values()) <= TOL_FP64


def test_isothermal_and_cosmological_terms(rhi):
    """Fixed temperature and a != 1, adot != 0 (1/a^3 and expansion terms)."""
    w = inputs.lognormal_hhe((10, 12, 14), box=150 * KPC, nsrc=2, dt=5e12, seed=5)
    w.theta = 1.0
    w.u_E = 1e-18
    a, adot = 0.4, 0.4 * 3e-17
    s = rhi.solver_for_workload(w, isothermal=1)
    p = oracle_problem(w, isothermal=True)
    ref = w.state()
    for _ in range(2):
        s.step(w.dt, a, adot, newton_tol=TIGHT_NEWTON_TOL, lin_tol=1e-12)
        ref, st = sv.implicit_step(p, ref, w.dt, a, adot, TIGHT_NEWTON_TOL)
        assert st["converged"]
    err = _field_errors(s.get_state(), ref, w)
    assert max(err.values()) <= TOL_FP64, err


def test_element_conservation_to_roundoff(rhi):
    """n_HI + n_HII = n_H and n_HeI + n_HeII + n_HeIII = n_He hold with every derived
    density non-negative, whatever the linear tolerance (the analogue of Table conservation)."""
    w = WL["lognormal_hhe"]
    for lin_tol in (1e-2, 1e-12):
        s = rhi.solver_for_workload(w)
        for _ in range(2):
            s.step(w.dt, newton_tol=1e-9, lin_tol=lin_tol)
        out = s.get_state()
        nH = w.nH.ravel()
        nHe = w.y_he * nH
        nHI, nHeI, nHeII = out["n"]
        assert np.all(nHI >= 0) and np.all(nH - nHI >= 0)
        assert np.all(nHeI >= 0) and np.all(nHeII >= 0) and np.all(nHe - nHeI - nHeII >= 0)


def test_precond_is_symmetric_and_positive(rhi):
    """One V-cycle is a symmetric positive definite operator (needed by CG)."""
    w = WL["lognormal_hhe"]
    for code in (rhi.RHI_PRECOND_MG_FP64, rhi.RHI_PRECOND_MG_FP32):
        s = rhi.solver_for_workload(w, precond=code, mg_levels=4)
        s.linearize(w.dt)
        rng = np.random.default_rng(0)
        a, b = rng.standard_normal(w.N), rng.standard_normal(w.N)
        Ma, Mb = s.precond_apply(a), s.precond_apply(b)
        rel = abs(b @ Ma - a @ Mb) / np.sqrt((a @ Ma) * (b @ Mb))
        assert rel < (1e-12 if code == rhi.RHI_PRECOND_MG_FP64 else 1e-5)
        assert a @ Ma > 0 and b @ Mb > 0


def test_argument_and_state_errors(rhi):
    w = inputs.uniform_h(4)
    p = rhi.params_for_workload(w)
    with pytest.raises(rhi.RhiError) as e:
        rhi.Solver(0, 4, 4, w.dx, p)
    assert e.value.code == rhi.RHI_ERR_ARG
    with pytest.raises(rhi.RhiError) as e:
        rhi.Solver(4, 4, 4, w.dx, p, bc=(1, 0, 0, 0, 0, 0))       # unpaired periodic face
    assert e.value.code == rhi.RHI_ERR_ARG
    s = rhi.Solver(4, 4, 4, w.dx, p)
    with pytest.raises(rhi.RhiError) as e:
        s.step(1e12)
    assert e.value.code == rhi.RHI_ERR_STATE
    st = w.state()
    bad = st["E"].copy()
    bad[5] = -1.0
    with pytest.raises(rhi.RhiError) as e:
        s.set_state(bad, st["e"], st["n"].ravel().copy(), w.nH.ravel().copy())
    assert e.value.code == rhi.RHI_ERR_NONPHYSICAL
    with pytest.raises(rhi.RhiError) as e:
        s.set_sources([[4, 0, 0]], [1e48])
    assert e.value.code == rhi.RHI_ERR_ARG


def test_nonconvergence_leaves_state_unchanged(rhi):
    """max_newton = 1 with a tolerance no single iteration meets: RHI_ERR_NONCONVERGED and the
    state stays at U^n."""
    w = WL["lognormal_hhe"]
    s = rhi.solver_for_workload(w, max_newton=1)
    before = s.get_state()
    rc = s.step(w.dt, newton_tol=1e-14, lin_tol=1e-3, check=False)
    assert rc == rhi.RHI_ERR_NONCONVERGED
    after = s.get_state()
    for k in ("E", "e", "n"):
        np.testing.assert_array_equal(before[k], after[k])


def test_faint_field_matches_oracle(rhi):
    """Half of the box starts with a radiation field 1e180 below the rest (E near 1e-200), as
    deep neutral gas reaches after many absorbing steps.  There the limiter's squares and
    1 / den^2 leave the FP64 range unless the face is rescaled (0 / 0 at the first residual).
    The step with the exact Newton matrix must stay finite and positive and match the oracle,
    which works with R = |dE| / (a dx Ebar) directly."""
    w = inputs.lognormal_hhe((10, 12, 14), box=200 * KPC, nsrc=2, dt=5e12, nsteps=1, seed=4)
    w.theta = 1.0
    w.u_E = 1e-18
    E = w.E.copy()
    E[: w.nz // 2] *= 1e-180
    w.E = E
    s = rhi.solver_for_workload(w, limiter_jacobian=2)
    s.step(w.dt, newton_tol=TIGHT_NEWTON_TOL, lin_tol=1e-12)
    got = s.get_state()
    s.close()
    p = oracle_problem(w)
    ref, _ = sv.implicit_step(p, w.state(), w.dt, 1.0, 0.0, TIGHT_NEWTON_TOL)
    Eg = np.asarray(got["E"]).reshape(w.nz, w.ny, w.nx)
    assert np.all(np.isfinite(Eg)) and np.all(Eg > 0)
    err = _field_errors(got, ref, w)
    assert max(err.values()) <= TOL_FP64, err
    # the faint half on its own: the floor then scales with the faint half's own maximum
    faint = np.zeros((w.nz, w.ny, w.nx), dtype=bool)
    faint[: w.nz // 2] = True
    err = _field_errors(got, ref, w, mask=faint)
    assert max(err.values()) <= TOL_FP64, err


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 7), (3, 1, 2)])
def test_degenerate_grids(rhi, shape):
    """A single cell and line / plane grids (diffusion with fewer than three axes)."""
    w = inputs.lognormal_hhe(shape, box=100 * KPC, nsrc=1, dt=5e12, seed=2)
    w.theta = 1.0
    w.u_E = 1e-18
    s = rhi.solver_for_workload(w)
    s.step(w.dt, newton_tol=TIGHT_NEWTON_TOL, lin_tol=1e-12)
    p = oracle_problem(w)
    ref, _ = sv.implicit_step(p, w.state(), w.dt, 1.0, 0.0, TIGHT_NEWTON_TOL)
    assert max(_field_errors(s.get_state(), ref, w).values()) <= TOL_FP64


def test_vcycle_graph_matches_direct_launches(rhi):
    """The FP32 V-cycle replayed as a CUDA graph runs the same kernels in the same order as the
    direct launches: steps and preconditioner applications agree bit for bit, also when the
    step size changes (the graph is captured again for the new dt theta) and when a profiled
    step in between runs the direct launches."""
    w = WL["lognormal_hhe"]
    out = []
    for graph in (0, 1):
        s = rhi.solver_for_workload(w, precond=rhi.RHI_PRECOND_MG_FP32, mg_levels=4,
                                    limiter_jacobian=2, vcycle_graph=graph)
        for k, dt in enumerate((w.dt, w.dt, 0.5 * w.dt)):
            if k == 1:
                s.set_profiling(True)
            s.step(dt, newton_tol=1e-10, lin_tol=1e-10)
            s.set_profiling(False)
        st = s.get_state()
        lin = s.linearize(w.dt)
        z = s.precond_apply(np.random.default_rng(0).standard_normal(s.N))
        out.append((st, lin["rhs"], z))
        s.close()
    for key in ("E", "e", "n"):
        assert np.array_equal(np.asarray(out[0][0][key]), np.asarray(out[1][0][key])), key
    assert np.array_equal(out[0][2], out[1][2])


@pytest.mark.parametrize("precond", ["mg32", "mg64"])
def test_krylov_graph_matches_direct_launches(rhi, precond):
    """BiCGStab as one CUDA graph launch per solve (a while node whose iterations decide on the
    device whether to continue) against the same kernels launched from the host with one read
    per iteration: the steps agree bit for bit, with the same Newton, Krylov and V-cycle
    counts, also across a change of step size (a new graph).  With the graph a step reads the
    device once at its start, once per Newton iteration (or line-search trial), and once at
    its end."""
    w = WL["lognormal_hhe"]
    code = {"mg32": rhi.RHI_PRECOND_MG_FP32, "mg64": rhi.RHI_PRECOND_MG_FP64}[precond]
    out = []
    for graph in (0, 1):
        s = rhi.solver_for_workload(w, precond=code, mg_levels=4, limiter_jacobian=2,
                                    krylov_graph=graph)
        stats = []
        for dt in (w.dt, w.dt, 0.5 * w.dt):
            s.step(dt, newton_tol=1e-10, lin_tol=1e-10)
            stats.append(s.stats())
        out.append((s.get_state(), stats))
        s.close()
    for key in ("E", "e", "n"):
        assert np.array_equal(np.asarray(out[0][0][key]), np.asarray(out[1][0][key])), key
    for a, b in zip(out[0][1], out[1][1]):
        for k in ("newton_its", "pcg_its", "vcycles", "backtracks", "krylov_fallbacks"):
            assert a[k] == b[k], (k, a[k], b[k])
    for st in out[1][1]:
        assert st["krylov_fallbacks"] == 0
        assert st["host_syncs"] <= st["newton_its"] + st["backtracks"] + st["final_missed"] + 2, st
        assert st["host_syncs"] < out[0][1][0]["host_syncs"]


@pytest.mark.parametrize("precond,tol", [("mg32", 1e-8), ("mg32", TIGHT_NEWTON_TOL),
                                         ("mg64", 1e-8)])
def test_predicted_final_iterate_matches_full_evaluation(rhi, precond, tol):
    """predict_final: the trial iterate the quadratic model expects to end the iteration is
    evaluated for its residual alone (W only, no Jacobian or Schur system), and in full only
    when it did not converge.  The iterates are those of predict_final = 0 bit for bit, with
    the same counts; the residual-only kernels evaluate the same formulas for W and f, which
    the compiler may contract into FMAs differently (a product that the full kernels reuse),
    so the last ||f|| of a step agrees to rounding.  At least one prediction is made."""
    w = WL["lognormal_hhe"]
    code = {"mg32": rhi.RHI_PRECOND_MG_FP32, "mg64": rhi.RHI_PRECOND_MG_FP64}[precond]
    out = []
    for pf in (0, 1):
        s = rhi.solver_for_workload(w, precond=code, mg_levels=4, limiter_jacobian=2,
                                    predict_final=pf)
        stats = []
        for dt in (w.dt, w.dt, 0.5 * w.dt, w.dt):
            s.step(dt, newton_tol=tol, lin_tol=1e-10)
            stats.append(s.stats())
        out.append((s.get_state(), stats))
        s.close()
    for key in ("E", "e", "n"):
        assert np.array_equal(np.asarray(out[0][0][key]), np.asarray(out[1][0][key])), key
    for a, b in zip(out[0][1], out[1][1]):
        for k in ("newton_its", "pcg_its", "vcycles", "backtracks"):
            assert a[k] == b[k], (k, a[k], b[k])
        assert np.allclose(a["res_history"], b["res_history"], rtol=1e-12, atol=0.0)
        assert a["res_history"][:a["newton_its"]] == b["res_history"][:b["newton_its"]]
        assert abs(a["res_final"] - b["res_final"]) <= 1e-12 * a["res_final"]
        assert a["final_predicted"] == 0
    pred = sum(st["final_predicted"] for st in out[1][1])
    missed = sum(st["final_missed"] for st in out[1][1])
    print(f"{precond}, tol {tol:g}: {pred} predicted final iterates, {missed} missed, "
          f"Newton its {[st['newton_its'] for st in out[1][1]]}")
    assert pred >= 1
