"""Learned Newton initial guess: the CUDA kernels (features, targets, BF16 tensor-core forward,
FP32 backward, Adam) vs the FP64 oracle in oracle/mlp.py, and the guess inside the implicit
step (same root as the oracle's Newton solution, fewer Newton iterations once trained)."""
import numpy as np
import pytest

from conftest import oracle_problem
from oracle import mlp as om, model as md, solve as sv
from paper_0901_1110_gb300 import inputs
from parity import TIGHT_NEWTON_TOL, field_errors

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


def _workload(seed, shape=(20, 22, 24), nsteps=4):
    w = inputs.lognormal_hhe(shape, box=200 * KPC, nsrc=3, dt=5e12, nsteps=nsteps, seed=seed)
    w.theta = 1.0
    w.u_E = 1e-18
    return w


def _flat_state(st):
    return dict(E=np.ascontiguousarray(st["E"]).ravel(), e=np.ascontiguousarray(st["e"]).ravel(),
                n=np.ascontiguousarray(st["n"]).ravel())


def _normalised(w, X):
    """Weights with the input normalisation set from the training features."""
    d = om.unpack(w)
    d["mean"] = X.mean(axis=0)
    sd = X.std(axis=0)
    d["scale"] = np.where(sd > 1e-3, sd, 1.0)
    return om.pack(d)


def _trajectory(s, w, nsteps):
    """Features at U^n and targets of U^n -> U^{n+1} along nsteps GPU steps."""
    Xs, Ys = [], []
    for _ in range(nsteps):
        old = _flat_state(s.get_state())
        Xs.append(s.mlp_features(w.dt))
        s.step(w.dt, newton_tol=1e-10, lin_tol=1e-10)
        Ys.append(s.mlp_targets(old))
    return np.concatenate(Xs), np.concatenate(Ys)


@pytest.fixture(scope="module")
def trained(rhi):
    """A network trained on the GPU on a 4-step trajectory of seed 11."""
    import torch
    w = _workload(11)
    s = rhi.solver_for_workload(w, precond=rhi.RHI_PRECOND_MG_FP32, mg_levels=4)
    X, Y = _trajectory(s, w, w.nsteps)
    w0 = _normalised(om.init_weights(3), X).astype(np.float32)
    s.mlp_set_weights(w0)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y).cuda()
    losses = [s.mlp_train(Xd, Yd, epochs=1, batch=512, lr=2e-3)]
    for _ in range(5):
        losses.append(s.mlp_train(Xd, Yd, epochs=8, batch=512, lr=2e-3))
    return dict(w=s.mlp_get_weights(), X=X, Y=Y, losses=losses, workload=w)


def test_features_and_targets_match_oracle(rhi):
    """Features of the state at t^n and targets of one step (FP32 kernels from the FP64
    state) vs the oracle's FP64 definitions, element by element."""
    w = _workload(5)
    s = rhi.solver_for_workload(w)
    p = oracle_problem(w)
    st0 = w.state()
    X = s.mlp_features(w.dt, a=0.7)
    Xr = om.features(p, st0, w.dt, a=0.7)
    np.testing.assert_allclose(X, Xr, rtol=2e-6, atol=2e-5)
    old = _flat_state(s.get_state())
    s.step(w.dt, newton_tol=1e-10, lin_tol=1e-10)
    Y = s.mlp_targets(old)
    new = s.get_state()
    old_n = dict(E=old["E"], e=old["e"], n=old["n"].reshape(w.ns, -1))
    Yr = om.targets(p, old_n, new)
    np.testing.assert_allclose(Y, Yr, rtol=2e-6, atol=2e-5)
    # after a step the features carry its change, here for a next step of half the length
    X = s.mlp_features(0.5 * w.dt, a=0.7)
    Xr = om.features(p, new, 0.5 * w.dt, a=0.7, prev=old_n, dt_prev=w.dt)
    assert np.abs(Xr[:, 9:12]).max() > 1e-3
    np.testing.assert_allclose(X, Xr, rtol=2e-6, atol=2e-5)


def test_tensor_core_forward_matches_oracle(rhi):
    """BF16 weights and activations with FP32 accumulation vs the FP64 forward pass: each
    layer rounds its inputs and weights to 8 significant bits (relative 2^-9), so the output
    error stays at the percent level of the output scale; ragged row counts and the
    64-row tiles both covered."""
    rng = np.random.default_rng(0)
    w = _normalised(om.init_weights(7), rng.standard_normal((256, om.NIN)) * 3 + 1)
    s = rhi.Solver(2, 2, 2, 1.0, rhi.rhi_params_default(1))
    s.mlp_set_weights(w.astype(np.float32))
    w32 = s.mlp_get_weights()
    assert np.array_equal(w32, w.astype(np.float32))
    for n in (1, 31, 33, 1000, 4099):
        X = (rng.standard_normal((n, om.NIN)) * 3 + 1).astype(np.float32)
        Y = s.mlp_forward(X)
        Yr = om.forward(w32.astype(np.float64), X.astype(np.float64))
        scale = max(1.0, float(np.abs(Yr).max()))
        err = np.abs(Y - Yr)
        assert err.max() <= 3e-2 * scale, (n, err.max(), scale)
        assert np.median(err) <= 5e-3 * scale
    s.close()


def test_gradient_matches_oracle(rhi):
    """FP32 per-sample backward + deterministic weight-gradient reduction vs the FP64 oracle
    gradient (normwise 1e-4) and loss (1e-5), with a ragged sample count."""
    rng = np.random.default_rng(1)
    w = _normalised(om.init_weights(2), rng.standard_normal((64, om.NIN)))
    w32 = w.astype(np.float32)
    s = rhi.Solver(2, 2, 2, 1.0, rhi.rhi_params_default(1))
    s.mlp_set_weights(w32)
    for n in (1, 200, 3001):
        X = rng.standard_normal((n, om.NIN)).astype(np.float32)
        Y = rng.standard_normal((n, 6)).astype(np.float32)
        loss, g = s.mlp_loss_grad(X, Y)
        lr, gr = om.loss_and_grad(w32.astype(np.float64), X.astype(np.float64), Y.astype(np.float64))
        assert abs(loss / lr - 1) < 1e-5
        assert np.linalg.norm(g - gr) <= 1e-4 * np.linalg.norm(gr), n
        assert np.all(g[-2 * om.NIN:] == 0)
    s.close()


def test_training_reduces_loss_and_is_deterministic(rhi, trained):
    """Adam on the GPU lowers the loss of the trajectory data by a large factor, and two runs
    from the same weights on the same data give identical weights."""
    import torch
    L = trained["losses"]
    assert L[-1] < 0.1 * L[0], L
    X, Y = trained["X"][:3000], trained["Y"][:3000]
    w0 = _normalised(om.init_weights(4), X).astype(np.float32)
    outs = []
    for _ in range(2):
        s = rhi.Solver(2, 2, 2, 1.0, rhi.rhi_params_default(3))
        s.mlp_set_weights(w0)
        s.mlp_train(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), epochs=2, batch=256,
                    lr=1e-3)
        outs.append(s.mlp_get_weights())
        s.close()
    assert np.array_equal(outs[0], outs[1])
    # the GPU loss of the trained weights agrees with the oracle's
    lr_, _ = om.loss_and_grad(outs[0].astype(np.float64), X.astype(np.float64), Y.astype(np.float64))
    s = rhi.Solver(2, 2, 2, 1.0, rhi.rhi_params_default(3))
    s.mlp_set_weights(outs[0])
    lg, _ = s.mlp_loss_grad(X, Y)
    assert abs(lg / lr_ - 1) < 1e-5


def test_learned_guess_reaches_the_same_root(rhi, trained):
    """The implicit step started from the network's guess converges to the oracle's Newton
    solution (started from U^n, exact linear solves)."""
    w = trained["workload"]
    s = rhi.solver_for_workload(w, guess=rhi.RHI_GUESS_LEARNED, mlp_restart=0, mlp_retry=0)
    s.mlp_set_weights(trained["w"])
    p = oracle_problem(w)
    ref = w.state()
    used = []
    for _ in range(2):
        s.step(w.dt, newton_tol=TIGHT_NEWTON_TOL, lin_tol=1e-12)
        st = s.stats()
        used.append(st["guess_used"])
        assert st["res_guess_prev"] > 0
        ref, info = sv.implicit_step(p, ref, w.dt, 1.0, 0.0, TIGHT_NEWTON_TOL, linear="direct")
        assert info["converged"]
        err = field_errors(s.get_state(), ref, w.nH, w.y_he, scales=(w.u_e, w.u_n, w.u_E))
        assert max(err.values()) <= 1e-10, err
    assert rhi.RHI_GUESS_LEARNED in used, used


def test_learned_guess_needs_weights(rhi):
    w = _workload(5, shape=(4, 4, 4))
    s = rhi.solver_for_workload(w, guess=rhi.RHI_GUESS_LEARNED)
    with pytest.raises(rhi.RhiError):
        s.step(w.dt)
    with pytest.raises(rhi.RhiError):
        s.mlp_set_weights(np.zeros(10, dtype=np.float32))
    bad = np.zeros(rhi.RHI_MLP_NWEIGHTS, dtype=np.float32)       # scale 0
    with pytest.raises(rhi.RhiError):
        s.mlp_set_weights(bad)


def test_learned_guess_gain(rhi, trained):
    """What the trained network gains, measured and bounded: on its training realisation and
    on a held-out one (another seed) the guess starts Newton closer to the root than U^n in the
    first step (||f|| at the guess below ||f(U^n)||: 1.079x and 1.015x on a GB300), and the
    learned start, with its fallback to U^n and its restart, needs no more Newton iterations in
    total than U^n.  The measured numbers are printed."""
    out = {}
    for tag, w in (("train", trained["workload"]), ("held_out", _workload(23))):
        its, ratios = {}, []
        for guess in (rhi.RHI_GUESS_PREVIOUS, rhi.RHI_GUESS_LEARNED):
            s = rhi.solver_for_workload(w, guess=guess, precond=rhi.RHI_PRECOND_MG_FP32,
                                        mg_levels=4)
            if guess == rhi.RHI_GUESS_LEARNED:
                s.mlp_set_weights(trained["w"])
            n = 0
            for _ in range(w.nsteps):
                if guess == rhi.RHI_GUESS_LEARNED:
                    st0 = s.get_state()
                    U0 = np.zeros((s.ns + 2, s.N))
                    U0[1:1 + s.ns] = st0["n"]
                    U0[1 + s.ns] = st0["E"]
                    r0 = s.residual(U0, w.dt)[1]
                    rg = s.residual(s.mlp_guess(w.dt), w.dt)[1]
                    ratios.append(r0 / rg)
                s.step(w.dt, newton_tol=1e-10, lin_tol=1e-10)
                n += s.stats()["newton_its"]
            its[guess] = n
            s.close()
        out[tag] = (its, ratios)
        print(f"{tag}: Newton iterations (U^n, learned) = ({its[0]}, {its[2]}), "
              f"||f(U^n)|| / ||f(guess)|| per step = {np.round(ratios, 3).tolist()}")
        assert its[rhi.RHI_GUESS_LEARNED] <= its[rhi.RHI_GUESS_PREVIOUS], (tag, its)
    assert out["train"][1][0] > 1.0, out
    assert out["held_out"][1][0] > 1.0, out


def test_learned_start_restart_reaches_the_same_root(rhi, trained):
    """With mlp_restart = 1 a learned start that needs more than one iteration is abandoned
    for U^n; the step still reaches the oracle's solution."""
    w = trained["workload"]
    s = rhi.solver_for_workload(w, guess=rhi.RHI_GUESS_LEARNED, mlp_restart=1)
    s.mlp_set_weights(trained["w"])
    s.step(w.dt, newton_tol=TIGHT_NEWTON_TOL, lin_tol=1e-12)
    st = s.stats()
    p = oracle_problem(w)
    ref, info = sv.implicit_step(p, w.state(), w.dt, 1.0, 0.0, TIGHT_NEWTON_TOL, linear="direct")
    err = field_errors(s.get_state(), ref, w.nH, w.y_he, scales=(w.u_e, w.u_n, w.u_E))
    assert max(err.values()) <= 1e-10, err
    if st["guess_restarts"]:
        assert st["guess_used"] == rhi.RHI_GUESS_PREVIOUS


def test_decoded_guess_matches_oracle_decode(rhi, trained):
    """The guess the step starts from (features, tensor-core forward and decode fused in one
    kernel) vs the oracle's FP64 decode of the same network outputs, with the change gate and
    the out-of-distribution gate; cells within float rounding of either threshold excluded."""
    w = _workload(29)
    p = oracle_problem(w)
    st = w.state()
    E0 = np.asarray(st["E"]).ravel()
    for gate, ood in ((0.0, 0.0), (0.05, 0.0), (0.0, 2.0), (1e-3, 6.0)):
        s = rhi.solver_for_workload(w, mlp_gate=gate, mlp_ood=ood)
        s.mlp_set_weights(trained["w"])
        X = s.mlp_features(w.dt)
        Y = s.mlp_forward(X).astype(np.float64)
        G = s.mlp_guess(w.dt)
        wts = trained["w"].astype(np.float64)
        X64 = X.astype(np.float64)
        mask = om.out_of_distribution(wts, X64, ood)
        ref = om.decode(p, st, Y, gate=gate, ood_mask=mask)
        # skip cells whose keep decision changes within a small margin of either threshold
        keep = lambda g, o: om.decode(p, st, Y, gate=g,
                                      ood_mask=om.out_of_distribution(wts, X64, o))["E"] == E0
        ok = (keep(max(gate - 1e-4, 0.0), ood * (1 + 1e-4)) ==
              keep(gate + 1e-4, ood * (1 - 1e-4) if ood > 0 else 0.0))
        assert ok.mean() > 0.95
        eh = np.asarray(st["e"]).ravel()
        # the decode's exponentials run in FP32 (relative error a few 1e-7); the guess only
        # starts Newton, whose root does not depend on it
        np.testing.assert_allclose((eh + G[0])[ok], ref["e"][ok], rtol=2e-6)
        np.testing.assert_allclose(G[1 + p.ns][ok], ref["E"][ok], rtol=2e-6)
        nref = np.asarray(ref["n"]).reshape(p.ns, -1)
        for X_ in range(p.ns):
            np.testing.assert_allclose(G[1 + X_][ok], nref[X_][ok], rtol=2e-6,
                                       atol=1e-12 * p.nH.max())
        assert np.all(G[1 + p.ns] > 0) and np.all(eh + G[0] > 0)
        if ood == 2.0:
            assert mask.any()
        s.close()


def test_residual_at_an_iterate_matches_oracle(rhi):
    """rhi_residual: f(U) at U^n and at a perturbed iterate vs the oracle's residual."""
    w = _workload(31, shape=(9, 10, 11))
    p = oracle_problem(w)
    st = w.state()
    s = rhi.solver_for_workload(w)
    Un = md.state_to_U(p, st)
    eh = np.asarray(st["e"]).ravel()
    rng = np.random.default_rng(0)
    U1 = Un.copy()
    U1[0] = 0.05 * eh * rng.standard_normal(p.N)
    U1[1:] *= 1.0 + 0.05 * rng.random((p.nv - 1, p.N))
    nHe = p.y_he * p.nH
    U1[2:4] = np.minimum(U1[2:4], 0.49 * nHe)
    g = md.build_g(p, Un, eh, w.dt, 1.0, 0.0)
    for U in (Un, U1):
        f, nrm = s.residual(U, w.dt)
        fr = md.residual(p, U, g, eh, w.dt, 1.0, 0.0) / p.scales()[:, None]
        scale = np.abs(fr).max()
        assert np.abs(f - fr).max() <= 1e-10 * scale
        assert abs(nrm / md.rms_norm(p, fr * p.scales()[:, None]) - 1) < 1e-10


def test_rejected_guess_skips_the_network_for_mlp_retry_steps(rhi):
    """An untrained network's guess loses to U^n; the next mlp_retry steps start from U^n
    without evaluating it, and the step after that tries it again."""
    w = _workload(7, shape=(10, 11, 12), nsteps=4)
    s = rhi.solver_for_workload(w, guess=rhi.RHI_GUESS_LEARNED, mlp_retry=2, mlp_gate=0.0,
                                mlp_ood=0.0)
    rng = np.random.default_rng(5)
    wts = om.init_weights(9)
    d = om.unpack(wts)
    d["b4"] = rng.normal(0.0, 3.0, om.NOUT)           # large random changes: a bad guess
    s.mlp_set_weights(om.pack(d).astype(np.float32))
    tried = []
    for _ in range(4):
        s.step(w.dt, newton_tol=1e-10, lin_tol=1e-10)
        st = s.stats()
        assert st["guess_used"] == rhi.RHI_GUESS_PREVIOUS
        tried.append(st["res_guess_prev"] > 0)
    assert tried == [True, False, False, True], tried
