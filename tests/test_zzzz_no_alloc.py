"""The allocation-free RMS norm against the library's own residual norm.

rhi_rms_norm_noalloc serves callers that may not allocate device memory (code running under
CUDA stream capture, where cudaMalloc is not allowed, or applications that own all device
memory through their own pool): its reduction scratch is a static device array.  It must give
the norm of eq. rmsnorm that rhi_implicit_step reports for the same residual, call after call
(the scratch keeps the previous call's contents)."""
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-10          # the FP64 parity tolerance of the GPU tests


def test_noalloc_norm_matches_the_step_residual_norm():
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    from paper_0901_1110_gb300 import _build
    _build.build()
    import paper_0901_1110_gb300 as rhi
    from paper_0901_1110_gb300 import inputs

    w = inputs.lognormal_hhe((18, 20, 24), box=200 * inputs.KPC, nsrc=3, dt=5e12)
    w.theta = 1.0
    w.u_E = 1e-18
    s = rhi.solver_for_workload(w, max_newton=0)
    lin = s.linearize(w.dt)                       # scaled residual f(U^n)
    # the existing entry point: a step with no Newton iteration reports ||f(U_0 = U^n)||
    rc = s.step(w.dt, newton_tol=1e-300, lin_tol=1e-10, check=False)
    assert rc == rhi.RHI_ERR_NONCONVERGED
    ref = s.stats()["res_initial"]
    assert ref > 0

    f = torch.from_numpy(lin["f"].ravel().copy()).cuda()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):                            # two calls in a row share the scratch
        out.fill_(-1.0)
        rc = rhi.rhi_rms_norm_noalloc(f.data_ptr(), f.numel(), f.numel(), out.data_ptr(), stream)
        assert rc == rhi.RHI_OK
        torch.cuda.synchronize()
        assert abs(out.item() / ref - 1.0) < TOL

    # a size beyond the scratch is refused before any launch
    rc = rhi.rhi_rms_norm_noalloc(f.data_ptr(), rhi.RHI_NOALLOC_MAX_COUNT + 1, 1,
                                  out.data_ptr(), stream)
    assert rc == rhi.RHI_ERR_ARG
    s.close()
