"""Pins of the oracle MLP (the learned Newton initial guess): gradients against finite
differences, and the target encoding against its decoding."""
import numpy as np

from conftest import oracle_problem
from oracle import mlp, solve as sv
from paper_0901_1110_gb300 import inputs


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    w = mlp.init_weights(3)
    d = mlp.unpack(w)
    d["mean"] = rng.standard_normal(mlp.NIN)
    d["scale"] = rng.uniform(0.5, 2.0, mlp.NIN)
    w = mlp.pack(d)
    X = rng.standard_normal((40, mlp.NIN))
    Y = rng.standard_normal((40, mlp.NOUT))
    loss, g = mlp.loss_and_grad(w, X, Y)
    trainable = mlp.NWEIGHTS - 2 * mlp.NIN
    idx = rng.choice(trainable, 300, replace=False)
    for i in idx:
        h = 1e-6 * max(1.0, abs(w[i]))
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (mlp.loss_and_grad(wp, X, Y)[0] - mlp.loss_and_grad(wm, X, Y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), (i, fd, g[i])
    assert np.all(g[trainable:] == 0.0)


def test_targets_decode_to_the_new_state():
    """decode(targets(old -> new)) reproduces new: the encoding loses nothing."""
    w = inputs.lognormal_hhe((5, 6, 7), box=100 * inputs.KPC, nsrc=2, dt=5e12)
    w.theta = 1.0
    w.u_E = 1e-18
    p = oracle_problem(w)
    old = w.state()
    new, _ = sv.implicit_step(p, old, w.dt, 1.0, 0.0, 1e-10)
    Y = mlp.targets(p, old, new)
    back = mlp.decode(p, old, Y)
    for k in ("E", "e", "n"):
        np.testing.assert_allclose(back[k], new[k], rtol=1e-10, atol=1e-14 * np.abs(new[k]).max())


def test_gate_keeps_quiet_cells():
    w = inputs.lognormal_hhe((4, 4, 4), nsrc=1)
    p = oracle_problem(w)
    st = w.state()
    Y = mlp.targets(p, st, st)                    # no change at all
    Y[:, 0] += 1e-4                               # a change below the gate
    out = mlp.decode(p, st, Y, gate=1e-3)
    np.testing.assert_array_equal(out["E"], st["E"])


def test_features_of_a_known_cell():
    w = inputs.uniform_h(2, x0=0.25, T0=100.0)
    p = oracle_problem(w, u_E=1e-20, u_n=1e-3)
    X = mlp.features(p, w.state(), 1e12)
    np.testing.assert_allclose(X[:, 0], 0.0, atol=1e-15)            # E = u_E
    np.testing.assert_allclose(X[:, 2], np.log10(0.75), rtol=1e-15)
    np.testing.assert_allclose(X[:, 5], 0.0, atol=1e-15)
    np.testing.assert_allclose(X[:, 8], 0.0, atol=1e-15)
    np.testing.assert_array_equal(X[:, 9:13], 0.0)                   # no previous step
    # a previous step with half the field, a quarter more gas energy, x_HI from 0.5 to 0.75,
    # and twice the step length
    st = w.state()
    prev = dict(E=st["E"] * 0.5, e=st["e"] * 1.25, n=st["n"] * (0.5 / 0.75))
    X = mlp.features(p, st, 1e12, prev=prev, dt_prev=2e12)
    np.testing.assert_allclose(X[:, 9], np.log10(2.0), rtol=1e-15)
    np.testing.assert_allclose(X[:, 10], -np.log10(1.25), rtol=1e-14)
    np.testing.assert_allclose(X[:, 11], np.log(3.0), rtol=1e-14)       # logit 3/4 - logit 1/2
    np.testing.assert_allclose(X[:, 12], -np.log10(2.0), rtol=1e-15)


def test_out_of_distribution_cells_keep_the_old_state():
    """A feature 7 scales from the training mean flags its cell; flagged cells decode to the
    old state whatever the outputs, the others follow the outputs."""
    w = inputs.lognormal_hhe((4, 4, 4), nsrc=1)
    p = oracle_problem(w)
    st = w.state()
    X = mlp.features(p, st, 5e12)
    d = mlp.unpack(mlp.init_weights(0))
    d["mean"] = X.mean(axis=0)
    d["scale"] = np.ones(mlp.NIN)
    wts = mlp.pack(d)
    Xo = X.copy()
    Xo[5, 3] = d["mean"][3] + 7.0
    Xo[9, 0] = d["mean"][0] - 7.0
    mask = mlp.out_of_distribution(wts, Xo, 6.0)
    expected = mlp.out_of_distribution(wts, X, 6.0)
    expected[[5, 9]] = True
    np.testing.assert_array_equal(mask, expected)
    assert not mlp.out_of_distribution(wts, Xo, 0.0).any()
    Y = mlp.targets(p, st, st)
    Y[:, 0] += 0.5                                  # every cell predicts E x 10^0.5
    out = mlp.decode(p, st, Y, gate=0.0, ood_mask=mask)
    E0 = np.asarray(st["E"]).ravel()
    np.testing.assert_array_equal(out["E"][mask], E0[mask])
    np.testing.assert_allclose(out["E"][~mask], E0[~mask] * 10 ** 0.5, rtol=1e-14)
