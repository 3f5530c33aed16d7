"""Oracle of the learned Newton initial guess: FP64 forward / backward of the per-cell MLP.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Not part of the paper: an added form in which a small network, trained on Newton solutions
the method itself produces, supplies the Newton initial guess U_0 (Sec. 3.2 leaves U_0 free;
Sec. 3.2.4 uses an explicit predictor).  The network maps 13 features of a cell at t^n (and of
its change over the previous step t^{n-1} -> t^n) to 6 outputs that fix the predicted state at
t^{n+1}:

  features  f0 = log10(E / u_E)          f1 = log10(e / u_e)       f2 = log10(n_HI / n_H)
            f3 = log10(n_HeI / n_He)     f4 = log10(n_HeII / n_He) f5 = log10(n_H / u_n)
            f6 = log10(dt Gamma_HI + 1e-30)   (ionisations per atom in one step)
            f7 = log10(1 + 4 pi eta dt / E)   (local source over field)
            f8 = log10(dt / 1e12 s)
            f9 = log10(E / E^{n-1})    f10 = log10(e / e^{n-1})
            f11 = logit x_HI - logit x_HI^{n-1}   (the previous step's change)
            f12 = log10(dt / dt^{n-1})            (this step over the previous one)
            (species fractions floored at 1e-30, x_HI in [1e-30, 1 - 1e-16] for the logits;
            H-only runs set f3 = f4 = 0; without a previous step f9..f12 = 0)
  outputs   o0 = log10(E' / E)   o1 = log10(e' / e)   o2 = logit(n_HI' / n_H)
            o3..o5 = logits of the He fractions (HeI, HeII, HeIII) under a softmax
  network   13 -> 64 -> 64 -> 64 -> 6, SiLU after the three hidden layers, inputs normalised
            as (f - mean) / scale.

Weight vector layout (shared with the library's C ABI): W1 (64x13, row major), b1 (64),
W2 (64x64), b2, W3 (64x64), b3, W4 (6x64), b4 (6), mean (13), scale (13).
"""
import numpy as np

from . import closure as cl

NIN, NHID, NOUT = 13, 64, 6
SHAPES = [("W1", (NHID, NIN)), ("b1", (NHID,)), ("W2", (NHID, NHID)), ("b2", (NHID,)),
          ("W3", (NHID, NHID)), ("b3", (NHID,)), ("W4", (NOUT, NHID)), ("b4", (NOUT,)),
          ("mean", (NIN,)), ("scale", (NIN,))]
NWEIGHTS = sum(int(np.prod(s)) for _, s in SHAPES)
FLOOR = 1e-30


def unpack(w):
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(w[o:o + n], dtype=np.float64).reshape(shape)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def init_weights(seed=0):
    """He-style random initialisation, zero biases, identity normalisation."""
    rng = np.random.default_rng(seed)
    d = {}
    for name, shape in SHAPES:
        if name.startswith("W"):
            d[name] = rng.standard_normal(shape) * np.sqrt(2.0 / shape[1])
        elif name == "scale":
            d[name] = np.ones(shape)
        else:
            d[name] = np.zeros(shape)
    return pack(d)


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def _logit_hi(n, nH):
    x = np.clip(n / nH, FLOOR, 1.0 - 1e-16)
    return np.log(x) - np.log1p(-x)


def features(p, state, dt, a=1.0, prev=None, dt_prev=None):
    """The 13 input features of every cell of ``p`` (oracle Problem) at the given state, with
    the previous step's state ``prev`` (E, e, n) and length ``dt_prev`` (None: no previous
    step)."""
    E = np.asarray(state["E"]).ravel()
    e = np.asarray(state["e"]).ravel()
    n = np.asarray(state["n"]).reshape(p.ns, -1)
    nH = p.nH
    nHe = p.y_he * nH
    X = np.empty((p.N, NIN))
    X[:, 0] = np.log10(E / p.u_E)
    X[:, 1] = np.log10(e / p.u_e)
    X[:, 2] = np.log10(np.maximum(n[0] / nH, FLOOR))
    if p.ns == 3:
        X[:, 3] = np.log10(np.maximum(n[1] / nHe, FLOOR))
        X[:, 4] = np.log10(np.maximum(n[2] / nHe, FLOOR))
    else:
        X[:, 3] = 0.0
        X[:, 4] = 0.0
    X[:, 5] = np.log10(nH / p.u_n)
    gam = cl.C_LIGHT * p.grey["pgam"][0] * E / a ** 3
    X[:, 6] = np.log10(dt * gam + FLOOR)
    X[:, 7] = np.log10(1.0 + p.src * dt / E)
    X[:, 8] = np.log10(dt / 1e12)
    X[:, 9:13] = 0.0
    if prev is not None:
        E0 = np.asarray(prev["E"]).ravel()
        e0 = np.asarray(prev["e"]).ravel()
        n0 = np.asarray(prev["n"]).reshape(p.ns, -1)
        X[:, 9] = np.log10(E / E0)
        X[:, 10] = np.log10(e / e0)
        X[:, 11] = _logit_hi(n[0], nH) - _logit_hi(n0[0], nH)
        X[:, 12] = np.log10(dt / dt_prev)
    return X


def targets(p, old, new):
    """The 6 training targets of every cell for the step old -> new (inverse of ``decode``)."""
    n0 = np.asarray(old["n"]).reshape(p.ns, -1)
    n1 = np.asarray(new["n"]).reshape(p.ns, -1)
    Y = np.zeros((p.N, NOUT))
    Y[:, 0] = np.log10(np.asarray(new["E"]).ravel() / np.asarray(old["E"]).ravel())
    Y[:, 1] = np.log10(np.asarray(new["e"]).ravel() / np.asarray(old["e"]).ravel())
    x = np.clip(n1[0] / p.nH, FLOOR, 1.0 - 1e-16)
    Y[:, 2] = np.log(x) - np.log1p(-x)
    if p.ns == 3:
        nHe = p.y_he * p.nH
        f = np.stack([n1[1], n1[2], nHe - n1[1] - n1[2]]) / nHe
        lf = np.log(np.maximum(f, FLOOR))
        Y[:, 3:6] = (lf - lf.mean(axis=0)).T
    return Y


def forward(w, X, keep=False):
    """Network outputs for inputs X (n, 9); with keep, also the pre-activations."""
    d = unpack(w)
    h0 = (X - d["mean"]) / d["scale"]
    z1 = h0 @ d["W1"].T + d["b1"]
    h1 = silu(z1)
    z2 = h1 @ d["W2"].T + d["b2"]
    h2 = silu(z2)
    z3 = h2 @ d["W3"].T + d["b3"]
    h3 = silu(z3)
    out = h3 @ d["W4"].T + d["b4"]
    if keep:
        return out, (h0, z1, h1, z2, h2, z3, h3)
    return out


def loss_and_grad(w, X, Y):
    """Mean squared error over samples and outputs, and its gradient wrt the weights (the
    normalisation entries get zero gradient)."""
    d = unpack(w)
    out, (h0, z1, h1, z2, h2, z3, h3) = forward(w, X, keep=True)
    m = X.shape[0]
    diff = out - Y
    loss = float(np.sum(diff * diff) / (m * NOUT))
    g4 = 2.0 * diff / (m * NOUT)                       # d loss / d out
    grads = {"W4": g4.T @ h3, "b4": g4.sum(axis=0)}
    d3 = (g4 @ d["W4"]) * dsilu(z3)
    grads["W3"], grads["b3"] = d3.T @ h2, d3.sum(axis=0)
    d2 = (d3 @ d["W3"]) * dsilu(z2)
    grads["W2"], grads["b2"] = d2.T @ h1, d2.sum(axis=0)
    d1 = (d2 @ d["W2"]) * dsilu(z1)
    grads["W1"], grads["b1"] = d1.T @ h0, d1.sum(axis=0)
    grads["mean"] = np.zeros(NIN)
    grads["scale"] = np.zeros(NIN)
    return loss, pack(grads)


def out_of_distribution(w, X, ood):
    """Cells whose normalised features (X - mean) / scale leave [-ood, ood] in any component:
    the network has seen too few such cells to be trusted there (ood <= 0: none)."""
    if ood is None or ood <= 0:
        return np.zeros(X.shape[0], dtype=bool)
    d = unpack(w)
    return np.any(np.abs((X - d["mean"]) / d["scale"]) > ood, axis=1)


def decode(p, state, out, gate=0.0, ood_mask=None):
    """Predicted state (E, e, n) from network outputs; cells whose predicted changes are all
    below ``gate`` (in log10 / logit units), and cells flagged in ``ood_mask``, keep the old
    state."""
    E0 = np.asarray(state["E"]).ravel()
    e0 = np.asarray(state["e"]).ravel()
    n0 = np.asarray(state["n"]).reshape(p.ns, -1)
    E = E0 * 10.0 ** out[:, 0]
    e = e0 * 10.0 ** out[:, 1]
    xHI = 1.0 / (1.0 + np.exp(-out[:, 2]))
    n = np.empty_like(n0)
    n[0] = p.nH * xHI
    change = np.maximum(np.abs(out[:, 0]), np.abs(out[:, 1]))
    x0 = np.clip(n0[0] / p.nH, FLOOR, 1.0 - 1e-16)
    change = np.maximum(change, np.abs(out[:, 2] - (np.log(x0) - np.log1p(-x0))))
    if p.ns == 3:
        nHe = p.y_he * p.nH
        z = out[:, 3:6] - out[:, 3:6].max(axis=1, keepdims=True)
        f = np.exp(z)
        f /= f.sum(axis=1, keepdims=True)
        n[1] = nHe * f[:, 0]
        n[2] = nHe * f[:, 1]
        f0 = np.stack([n0[1], n0[2], nHe - n0[1] - n0[2]]).T / nHe[:, None]
        dlog = np.abs(np.log(np.maximum(f, FLOOR)) - np.log(np.maximum(f0, FLOOR)))
        change = np.maximum(change, dlog.max(axis=1))
    keep = change < gate
    if ood_mask is not None:
        keep = keep | ood_mask
    E = np.where(keep, E0, E)
    e = np.where(keep, e0, e)
    n = np.where(keep[None, :], n0, n)
    return dict(E=E, e=e, n=n)
