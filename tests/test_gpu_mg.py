"""The multigrid preconditioner (Sec. 3.2.2: the Schur system in E is solved by multigrid-
preconditioned Krylov iterations) against the numpy restatement of the same V-cycle in
``mg_reference.py``.

The V-cycle is a fixed linear operator, so one application to a random vector pins every
multigrid kernel at once: the FP32 copy of the finest operator, the re-discretised coarse
operators, the weighted-Jacobi sweeps, the residual restriction, the prolongation and the
coarsest-level solve.  The restatement starts from the finest operator as the library exports
it (Schur diagonal and face entries of the lagged-D Newton matrix).
"""
import numpy as np
import pytest

import mg_reference as mgr
from paper_0901_1110_gb300 import inputs

pytestmark = pytest.mark.gpu
KPC = inputs.KPC


@pytest.fixture(scope="module")
def rhi():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_0901_1110_gb300 import _build
    _build.build()
    import paper_0901_1110_gb300 as rhi
    rhi.lib()
    return rhi


CASES = {
    # ragged extents: odd sizes on the coarser levels, 27 cells on the coarsest
    "lognormal_ragged": dict(shape=(18, 20, 24), bc=("zero_flux",) * 6, seed=0, levels=4),
    "lognormal_periodic": dict(shape=(8, 13, 16), bc=("periodic",) * 6, seed=3, levels=3),
    # rows of 256 cells and 16 planes: the FP32 finest-level sweeps run as the staged
    # (bulk-copy) kernel
    "wide_rows": dict(shape=(16, 6, 256), bc=("zero_flux",) * 6, seed=7, levels=3),
    "wide_rows_periodic": dict(shape=(16, 5, 256), bc=("periodic",) * 6, seed=8, levels=3),
}
# FP64: rounding order only; FP32: the cycle in single precision against the FP64 restatement
TOL = {"fp64": 1e-12, "fp32": 1e-4}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("matrix", ["lagged", "newton"])
def test_vcycle_matches_numpy_restatement(rhi, case, precision, matrix):
    """The hierarchy of the lagged-D matrix (symmetric), and that of the exact Newton matrix
    (non-symmetric: its faces carry both couplings, Wp from the exported upper entries)."""
    c = CASES[case]
    w = inputs.lognormal_hhe(c["shape"], box=200 * KPC, nsrc=3, dt=5e12, nsteps=2,
                             bc=c["bc"], seed=c["seed"])
    nz, ny, nx = w.nz, w.ny, w.nx
    w.theta = 1.0
    w.u_E = 1e-18
    code = rhi.RHI_PRECOND_MG_FP64 if precision == "fp64" else rhi.RHI_PRECOND_MG_FP32
    omega, pre, post, coarse = 0.9, 2, 2, 16
    s = rhi.solver_for_workload(w, precond=code, mg_levels=c["levels"], mg_pre=pre,
                                mg_post=post, mg_coarse_sweeps=coarse, mg_omega=omega,
                                limiter_jacobian=0 if matrix == "lagged" else 2, mg_matrix=1,
                                vcycle_graph=0)
    # a step first, so that the operator carries an ionised region around the sources
    s.step(w.dt, newton_tol=1e-9, lin_tol=1e-10)
    lin = s.linearize(w.dt)
    r = np.random.default_rng(5).standard_normal(s.N)
    z = s.precond_apply(r)
    s.close()
    shape = (nz, ny, nx)
    W = [lin["face"][ax].reshape(shape) for ax in range(3)]
    Wp = None
    if matrix == "newton":
        # row c's coupling to its upper neighbour sits, per face, at the upper cell
        Wp = [np.roll(lin["face_hi"][ax].reshape(shape), 1, axis=2 - ax) for ax in range(3)]
        assert max(np.abs(Wp[ax] - W[ax]).max() for ax in range(3)) > 1e-6 * np.abs(W[0]).max()
    ops = mgr.hierarchy(lin["diag"].reshape(shape), W, c["levels"], Wp)
    assert len(ops) == c["levels"]
    zr = mgr.vcycle(ops, r.reshape(shape), omega, pre, post, coarse).ravel()
    rel = np.linalg.norm(z - zr) / np.linalg.norm(zr)
    assert rel <= TOL[precision], rel
