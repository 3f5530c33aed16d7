"""The named workloads at their own sizes against the FP64 oracle, per element.

* The 32^3 hydrogen benchmark as it is specified: 1 Mpc comoving box, uniform n_H = 1e-3,
  T0 = 100 K, x_HII = 1e-4, one central 5e48 s^-1 source at 13.6 eV, zero-flux boundaries,
  a = 1, five steps of 1e12 s, theta = 1 (the step with theta = 0.51 has no positive
  solution there: c kappa dt = 189), Newton tolerance 1e-8 and Krylov tolerance 1e-10; and the
  same five steps at tight tolerances.
* A 64^3 sub-box of the 256^3 hydrogen + helium lognormal recipe at the timed run's cell size
  (1 Mpc / 256), with the timed run's settings (exact Newton matrix, BiCGStab, 6 multigrid
  levels, Newton tolerance 1e-8, Krylov tolerance 1e-10): the plain FP64 form, the mixed form
  (FP32 multigrid) and the learned + mixed form, each against the oracle converged to 1e-14.

At tight tolerances (both sides to 1e-14) the bound is the FP64 parity bound, 1e-10 per element
on E, e and every species fraction.  At the configured Newton tolerance 1e-8 the GPU stops
where ||f|| (eq. rmsnorm over the scaled unknowns) first falls below 1e-8.  That criterion
bounds the distance to the root in the scaled unknowns (E / u_E, e / u_e, n / u_n), not cell by
cell: a cell whose E is a millionth of u_E is held only to its share of the RMS norm.  These
tests hold the RMS of the scaled distance below 10 times the tolerance and its largest element
below sqrt(N (N_s + 2)) times the tolerance (what an RMS bound allows one element), and print
the per-element errors, which the bench line also reports.
"""
import time

import numpy as np
import pytest

from conftest import oracle_problem
from oracle import solve as sv
from paper_0901_1110_gb300 import inputs
from parity import TIGHT_NEWTON_TOL, field_errors, scaled_errors

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


def _scaled_ok(sc, w, tol):
    n_unknowns = w.N * (w.ns + 2)
    return sc["rms"] <= 10 * tol and max(sc[k] for k in ("E", "e", "n") if k in sc) <= np.sqrt(n_unknowns) * tol


@pytest.fixture(scope="module")
def rhi():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_0901_1110_gb300 import _build
    _build.build()
    import paper_0901_1110_gb300 as rhi
    rhi.lib()
    return rhi


@pytest.fixture(scope="module")
def config1_reference():
    """The oracle's five steps of the 32^3 benchmark, converged to 1e-14: exact Newton matrix,
    Schur complement, BiCGStab to 1e-14."""
    w = inputs.config_uniform_32()
    p = oracle_problem(w, limiter_jacobian="exact")
    ref, states = w.state(), []
    for _ in range(w.nsteps):
        ref, info = sv.implicit_step(p, ref, w.dt, 1.0, 0.0, TIGHT_NEWTON_TOL, linear="schur_cg")
        assert info["converged"]
        states.append(ref)
    return w, states


@pytest.mark.timeout(900)
@pytest.mark.parametrize("ljac", [0, 2])
@pytest.mark.parametrize("tols", [(1e-8, 1e-10), (TIGHT_NEWTON_TOL, 1e-12)])
def test_uniform_32_benchmark_as_stated(rhi, config1_reference, ljac, tols):
    w, states = config1_reference
    assert (w.nx, w.ny, w.nz) == (32, 32, 32) and w.nsteps == 5 and w.dt == 1e12
    s = rhi.solver_for_workload(w, precond=rhi.RHI_PRECOND_MG_FP64, limiter_jacobian=ljac)
    for k in range(w.nsteps):
        s.step(w.dt, 1.0, 0.0, newton_tol=tols[0], lin_tol=tols[1])
        st = s.stats()
        got = s.get_state()
        tight = tols[0] <= TIGHT_NEWTON_TOL
        # at tight tolerances the allowance of the Newton resolution; at the configured one the
        # raw per-element error, printed
        err = field_errors(got, states[k], w.nH, w.y_he,
                           scales=(w.u_e, w.u_n, w.u_E) if tight else None)
        sc = scaled_errors(got, states[k], (w.u_e, w.u_n, w.u_E), w.ns)
        print(f"32^3 step {k}: matrix {ljac}, tols {tols}: newton {st['newton_its']} "
              f"krylov {st['pcg_its']} per-element errors "
              + " ".join(f"{a}={b:.2e}" for a, b in err.items())
              + " scaled " + " ".join(f"{a}={b:.2e}" for a, b in sc.items()))
        if tight:
            assert max(err.values()) <= TOL_FP64, (k, err)
        else:
            assert _scaled_ok(sc, w, tols[0]), (k, sc)
    s.close()


def _subbox(n=64, seed=0):
    nsrc = max(1, round(64 * (n / 256) ** 3))
    return inputs.config_lognormal(n, nsrc=nsrc, seed=seed, box=inputs.MPC * n / 256)


NSTEPS_SUBBOX = 4


@pytest.fixture(scope="module")
def subbox_reference():
    """Four steps of the 64^3 sub-box by the oracle: exact Newton matrix, Schur complement and
    BiCGStab to 1e-14, Newton to 1e-14."""
    w = _subbox()
    p = oracle_problem(w, limiter_jacobian="exact")
    ref, states = w.state(), []
    t0 = time.perf_counter()
    for _ in range(NSTEPS_SUBBOX):
        ref, info = sv.implicit_step(p, ref, w.dt, 1.0, 0.0, TIGHT_NEWTON_TOL, linear="schur_cg")
        assert info["converged"], info["res_history"]
        states.append(ref)
    print(f"oracle 64^3 sub-box: {NSTEPS_SUBBOX} steps in {time.perf_counter() - t0:.1f} s")
    return w, states


def _train_small(rhi):
    """A learned guess trained on the GPU on six steps of a 32^3 sub-box of another seed."""
    import torch
    w = _subbox(32, seed=77)
    s = rhi.solver_for_workload(w, precond=rhi.RHI_PRECOND_MG_FP32, mg_levels=5,
                                limiter_jacobian=2)
    Xs, Ys = [], []
    for _ in range(6):
        st = s.get_state()
        old = dict(E=np.ascontiguousarray(st["E"]), e=np.ascontiguousarray(st["e"]),
                   n=np.ascontiguousarray(st["n"]).ravel())
        Xs.append(s.mlp_features(w.dt))
        s.step(w.dt, 1.0, 0.0, w.newton_tol, w.lin_tol)
        Ys.append(s.mlp_targets(old))
    X = np.concatenate(Xs)
    Y = np.concatenate(Ys)
    rng = np.random.default_rng(0)
    I, H, O = rhi.RHI_MLP_IN, rhi.RHI_MLP_HID, rhi.RHI_MLP_OUT
    parts = []
    for rows, cols in ((H, I), (H, H), (H, H), (O, H)):
        parts += [rng.standard_normal(rows * cols) * np.sqrt(2.0 / cols), np.zeros(rows)]
    sd = X.std(axis=0)
    parts += [X.mean(axis=0), np.where(sd > 1e-3, sd, 1.0)]
    s.mlp_set_weights(np.concatenate(parts).astype(np.float32))
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y).cuda()
    s.mlp_train(Xd, Yd, epochs=3, batch=4096, lr=2e-3)
    wts = s.mlp_get_weights()
    s.close()
    return wts


@pytest.mark.timeout(1800)
def test_bench_subbox_three_forms_match_oracle(rhi, subbox_reference):
    w, states = subbox_reference
    weights = _train_small(rhi)
    forms = {"plain_fp64": (rhi.RHI_PRECOND_MG_FP64, rhi.RHI_GUESS_PREVIOUS),
             "mixed_fp32mg": (rhi.RHI_PRECOND_MG_FP32, rhi.RHI_GUESS_PREVIOUS),
             "learned_mixed": (rhi.RHI_PRECOND_MG_FP32, rhi.RHI_GUESS_LEARNED)}
    for name, (pc, guess) in forms.items():
        s = rhi.solver_for_workload(w, precond=pc, mg_levels=6, theta=1.0, limiter_jacobian=2,
                                    max_newton=200, guess=guess)
        if guess == rhi.RHI_GUESS_LEARNED:
            s.mlp_set_weights(weights)
        worst, worst_sc = {}, {}
        for k in range(NSTEPS_SUBBOX):
            s.step(w.dt, 1.0, 0.0, w.newton_tol, w.lin_tol)
            got = s.get_state()
            for a, b in field_errors(got, states[k], w.nH, w.y_he).items():
                worst[a] = max(worst.get(a, 0.0), b)
            for a, b in scaled_errors(got, states[k], (w.u_e, w.u_n, w.u_E), w.ns).items():
                worst_sc[a] = max(worst_sc.get(a, 0.0), b)
        print(f"64^3 sub-box, {name}: worst over {NSTEPS_SUBBOX} steps, per element "
              + " ".join(f"{a}={b:.2e}" for a, b in worst.items())
              + "; scaled " + " ".join(f"{a}={b:.2e}" for a, b in worst_sc.items()))
        assert _scaled_ok(worst_sc, w, w.newton_tol), (name, worst_sc)
        s.close()


@pytest.mark.timeout(1800)
def test_bench_subbox_tight_tolerances_match_oracle(rhi, subbox_reference):
    """The same sub-box with the mixed form at tight tolerances meets the FP64 bound: the FP32
    multigrid changes only the preconditioner, not the root."""
    w, states = subbox_reference
    s = rhi.solver_for_workload(w, precond=rhi.RHI_PRECOND_MG_FP32, mg_levels=6, theta=1.0,
                                limiter_jacobian=2, max_newton=200)
    for k in range(NSTEPS_SUBBOX):
        s.step(w.dt, 1.0, 0.0, TIGHT_NEWTON_TOL, 1e-12)
        err = field_errors(s.get_state(), states[k], w.nH, w.y_he, scales=(w.u_e, w.u_n, w.u_E))
        assert max(err.values()) <= TOL_FP64, (k, err)
    s.close()
