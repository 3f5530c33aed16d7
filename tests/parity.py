"""The per-element bound every GPU-against-oracle comparison uses.

For each field, the largest over cells of |gpu - ref| / (|ref| + floor * max|ref|), with
floor = 1e-12.  A cell far below the brightest one is then held to its own magnitude, down to
twelve decades under the field's maximum, instead of to the field's maximum.

The species are compared as fractions of their element: x_HI = n_HI / n_H, x_HII = 1 - x_HI,
and for helium x_HeI, x_HeII and x_HeIII = 1 - x_HeI - x_HeII, each over n_He = y_he n_H.  An
ionised cell's small neutral fraction and a neutral cell's small ionised fraction are each held
to their own size.  The derived fractions are formed from the densities on each side in the
same way (n_HII = n_H - n_HI), as the library and the oracle form them.  Neither side holds a
derived density to better than the rounding of that subtraction, a unit in the last place of
the element total, so a derived fraction's difference is taken net of DERIVED_ULPS units of
2^-52 before the per-element bound applies.  (Two oracle solves that differ only in their last
Newton iterate differ by 2.2e-8 relative in an x_HeIII of 1e-8, which is 1 unit.)

Both sides solve f(U) = 0 to the Newton tolerance on the RMS norm of eq. rmsnorm, which does
not hold a faint cell to its own size: stopped at 1e-12, the oracle's own E differs from its
converged root by 8e-10 relative in the faintest cells of a lognormal box (D lagged, linear
convergence).  The FP64 comparisons therefore solve both sides to TIGHT_NEWTON_TOL, below which
the next Newton iterate is at the rounding floor.

Even there the stopping test fixes each unknown only to about TIGHT_NEWTON_TOL of its scale u
(u_E for E, u_e for e): a cell whose E is 10^-8 of u_E carries that rounding as 1e-6 of its own
value.  Two exact oracle solves of the same step that differ only in their Newton matrix (D
lagged with sparse LU, and the exact matrix with the Schur complement and BiCGStab), both to
1e-14, differ by 1e-9 relative in such cells, 3e-34 erg cm^-3 against u_E = 1e-17.  When the
scalings are given, E's and e's differences are therefore taken net of TIGHT_NEWTON_TOL u
before the per-element bound applies.
"""
import numpy as np

FLOOR = 1e-12
DERIVED_ULPS = 4.0
TIGHT_NEWTON_TOL = 1e-14


def rel_error(got, ref, floor=FLOOR, mask=None, allowance=0.0):
    """max |got - ref| / (|ref| + floor max|ref|) over the cells (of `mask`, when given); with
    an absolute allowance a, the difference is taken as max(|got - ref| - a, 0)."""
    g = np.asarray(got, dtype=np.float64).ravel()
    r = np.asarray(ref, dtype=np.float64).ravel()
    if g.shape != r.shape:
        raise ValueError(f"shape mismatch {g.shape} vs {r.shape}")
    if mask is not None:
        m = np.asarray(mask, dtype=bool).ravel()
        g, r = g[m], r[m]
    if r.size == 0:
        return 0.0
    den = np.abs(r) + floor * np.abs(r).max()
    d = np.maximum(np.abs(g - r) - allowance, 0.0)
    # a field that is exactly zero everywhere on both sides agrees
    ok = den > 0
    if not ok.all():
        if np.any(d[~ok] > 0):
            return float("inf")
        d, den = d[ok], den[ok]
    return float((d / den).max()) if d.size else 0.0


def fractions(n, nH, y_he):
    """Species fractions of both elements from the independent densities (ns x N)."""
    nH = np.asarray(nH, dtype=np.float64).ravel()
    n = np.asarray(n, dtype=np.float64).reshape(-1, nH.size)
    out = {}
    if n.shape[0] >= 1:
        out["x_HI"] = n[0] / nH
        out["x_HII"] = (nH - n[0]) / nH
    if n.shape[0] == 3:
        nHe = y_he * nH
        out["x_HeI"] = n[1] / nHe
        out["x_HeII"] = n[2] / nHe
        out["x_HeIII"] = (nHe - n[1] - n[2]) / nHe
    return out


def field_errors(got, ref, nH, y_he=0.0, mask=None, keys=("E", "e"), scales=None,
                 newton_tol=TIGHT_NEWTON_TOL):
    """Per-element error of E, e and every species fraction (dict name -> error).  scales =
    (u_e, u_n, u_E): E's and e's differences net of newton_tol u (the Newton iteration's
    resolution of that unknown)."""
    out = {}
    for k in keys:
        allow = 0.0
        if scales is not None:
            allow = newton_tol * (scales[2] if k == "E" else scales[0])
        out[k] = rel_error(got[k], ref[k], mask=mask, allowance=allow)
    if "n" in ref and np.asarray(ref["n"]).size:
        fg = fractions(got["n"], nH, y_he)
        fr = fractions(ref["n"], nH, y_he)
        for k in fr:
            derived = k in ("x_HII", "x_HeIII")
            out[k] = rel_error(fg[k], fr[k], mask=mask,
                               allowance=DERIVED_ULPS * 2.0 ** -52 if derived else 0.0)
    return out


def worst(errs):
    return max(errs.values()) if errs else 0.0


def scaled_errors(got, ref, scales, ns):
    """Distance in the scaled unknowns (E / u_E, e / u_e, n / u_n), whose RMS residual the
    Newton iteration stops on: the RMS over all N (N_s + 2) unknowns ("rms") and the largest
    one per field ("E", "e", "n")."""
    u_e, u_n, u_E = scales
    dE = (np.asarray(got["E"]).ravel() - np.asarray(ref["E"]).ravel()) / u_E
    de = (np.asarray(got["e"]).ravel() - np.asarray(ref["e"]).ravel()) / u_e
    parts = [dE, de]
    out = {"E": float(np.abs(dE).max()), "e": float(np.abs(de).max())}
    if ns:
        dn = (np.asarray(got["n"]).reshape(ns, -1) - np.asarray(ref["n"]).reshape(ns, -1)) / u_n
        out["n"] = float(np.abs(dn).max())
        parts += list(dn)
    allp = np.concatenate([np.ravel(q) for q in parts])
    out["rms"] = float(np.sqrt(np.mean(allp ** 2)))
    return out
