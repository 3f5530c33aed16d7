"""Parity at the full size of the bench: the 256^3 H + He lognormal workload (64 sources) in
the bench's launch configuration (exact Newton matrix, BiCGStab, FP32 multigrid with 6 levels,
theta = 1).  The oracle cannot solve 16.8 M cells, so

- it computes the cell-local rows of the residual of eq. nonlinear_residual (gas energy and
  species: rates, photoionisation and photoheating from the cell's own E) one sampled cell at
  a time, and these are compared with the GPU's residual at U^n;
- the step's result is checked for what holds at any size: finite, E > 0, e > 0, every
  species (independent and derived) within [0, element total] up to roundoff, and the final
  ||f|| of eq. rmsnorm below the Newton tolerance.

The cell-local method itself is pinned on the CPU against the oracle's full-grid residual.
"""
import numpy as np
import pytest

from conftest import oracle_problem
from oracle import closure as cl, model as md
from paper_0901_1110_gb300 import inputs

N_SAMPLE = 256


def _state_U(w, st):
    """Newton unknowns at t^n in the iterate layout of the C ABI: (e_c = 0, n, E)."""
    U = np.zeros((w.ns + 2, w.N))
    U[1:1 + w.ns] = np.asarray(st["n"]).reshape(w.ns, w.N)
    U[1 + w.ns] = np.asarray(st["E"]).ravel()
    return U


def _local_rows(w, Un, eh, src, cells, rates):
    """Scaled gas-energy and species rows of f(U^n) at the given cells, each cell as a
    one-cell oracle problem (no faces: the rows hold no diffusion).  src is flat over cells."""
    grey = cl.grey_constants(*w.spectrum, w.ns)
    nH = w.nH.ravel()
    src = np.asarray(src).ravel()
    out = np.empty((w.ns + 1, len(cells)))
    for j, c in enumerate(cells):
        p = md.Problem(nx=1, ny=1, nz=1, dx=w.dx, ns=w.ns, nH=nH[c:c + 1], src=src[c:c + 1],
                       grey=grey, y_he=w.y_he, theta=w.theta, u_e=w.u_e, u_n=w.u_n,
                       u_E=w.u_E, rates=rates)
        U = Un[:, c:c + 1]
        e1 = eh[c:c + 1]
        g = md.build_g(p, U, e1, w.dt, 1.0, 0.0)
        f = md.residual(p, U, g, e1, w.dt, 1.0, 0.0) / p.scales()[:, None]
        out[:, j] = f[:w.ns + 1, 0]
    return out


def test_local_rows_equal_full_grid_rows():
    """CPU pin of the sampled check: the one-cell rows equal the full-grid oracle's rows."""
    w = inputs.lognormal_hhe((6, 7, 8), box=200 * inputs.KPC, nsrc=3, dt=5e12, seed=2)
    w.theta = 1.0
    w.u_E = 1e-18
    p = oracle_problem(w)
    st = w.state()
    Un = _state_U(w, st)
    eh = np.asarray(st["e"]).ravel()
    g = md.build_g(p, Un, eh, w.dt, 1.0, 0.0)
    full = md.residual(p, Un, g, eh, w.dt, 1.0, 0.0) / p.scales()[:, None]
    cells = np.arange(w.N)
    local = _local_rows(w, Un, eh, p.src, cells, cl.RateTable())
    scale = np.abs(full[:w.ns + 1]).max()
    assert np.abs(local - full[:w.ns + 1]).max() <= 1e-13 * scale
    # the sources make some rows large and most small: the comparison is not trivial
    assert np.abs(full[:w.ns + 1]).max() > 1e3 * np.median(np.abs(full[:w.ns + 1]))


@pytest.fixture(scope="module")
def rhi():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_0901_1110_gb300 import _build
    _build.build()
    import paper_0901_1110_gb300 as rhi
    rhi.lib()
    return rhi


def _sample_cells(w, rng):
    """Random cells, every source cell, and cells around the sources (where one step ionises
    and heats the gas)."""
    cells = [rng.integers(0, w.N, N_SAMPLE)]
    ijk = np.asarray(w.src_ijk)
    for off in rng.integers(-8, 9, size=(4, 3)):
        q = np.clip(ijk + off, 0, [w.nx - 1, w.ny - 1, w.nz - 1])
        cells.append(q[:, 0] + w.nx * (q[:, 1] + w.ny * q[:, 2]))
    cells.append(ijk[:, 0] + w.nx * (ijk[:, 1] + w.ny * ijk[:, 2]))
    return np.unique(np.concatenate(cells).astype(np.int64))


@pytest.mark.gpu
def test_bench_size_residual_rows_and_step_properties(rhi):
    w = inputs.config_lognormal(256, nsrc=64, seed=0)
    s = rhi.solver_for_workload(w, precond=rhi.RHI_PRECOND_MG_FP32, mg_levels=6, theta=1.0,
                                limiter_jacobian=2, max_newton=200)
    grey = cl.grey_constants(*w.spectrum, w.ns)
    src = np.asarray(cl.deposit_sources(w.nH.shape, w.dx, w.src_ijk, w.src_rate,
                                        grey["eps"])).ravel()
    cells = _sample_cells(w, np.random.default_rng(17))
    rates = cl.RateTable()

    def check_rows(st):
        """GPU residual rows at U = (0, n, E) of state st (f = dt L(U), the state being
        U^n of the residual) against the one-cell oracle rows."""
        U = _state_U(w, st)
        eh = np.asarray(st["e"]).ravel()
        f, _ = s.residual(U, w.dt)
        ref = _local_rows(w, U, eh, src, cells, rates)
        got = f[:w.ns + 1, cells]
        assert np.abs(got - ref).max() <= 1e-10 * np.abs(ref).max()

    check_rows(w.state())
    # one step in the bench's configuration, then what holds at any size
    s.step(w.dt, 1.0, 0.0, w.newton_tol, w.lin_tol)
    stats = s.stats()
    out = s.get_state()
    E, e = np.asarray(out["E"]), np.asarray(out["e"])
    n = np.asarray(out["n"]).reshape(w.ns, w.N)
    assert np.all(np.isfinite(E)) and np.all(np.isfinite(e)) and np.all(np.isfinite(n))
    assert np.all(E > 0) and np.all(e > 0)
    nH = w.nH.ravel()
    nHe = w.y_he * nH
    nHI, nHeI, nHeII = n
    tinyH, tinyHe = 1e-13 * nH, 1e-13 * nHe
    for q, tiny in ((nHI, tinyH), (nH - nHI, tinyH), (nHeI, tinyHe), (nHeII, tinyHe),
                    (nHe - nHeI - nHeII, tinyHe)):
        assert np.all(q >= -tiny)
    assert stats["newton_its"] >= 1
    assert stats["res_history"][-1] < w.newton_tol
    # the same rows at the new state, with ionised and heated gas around the sources
    check_rows(dict(E=E, e=e, n=n))
    s.close()
