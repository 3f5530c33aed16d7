"""The per-element bound every GPU-against-oracle comparison uses.

For each field, the largest over cells of |gpu - ref| / (|ref| + floor * max|ref|), with
floor = 1e-12.  A cell far below the brightest one is then held to its own magnitude, down to
twelve decades under the field's maximum, instead of to the field's maximum.

The species are compared as fractions of their element: x_HI = n_HI / n_H, x_HII = 1 - x_HI,
and for helium x_HeI, x_HeII and x_HeIII = 1 - x_HeI - x_HeII, each over n_He = y_he n_H.  An
ionised cell's small neutral fraction and a neutral cell's small ionised fraction are each held
to their own size.  The derived fractions are formed from the densities on each side in the
same way (n_HII = n_H - n_HI), as the library and the oracle form them.
"""
import numpy as np

FLOOR = 1e-12


def rel_error(got, ref, floor=FLOOR, mask=None):
    """max |got - ref| / (|ref| + floor max|ref|) over the cells (of `mask`, when given)."""
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
    d = np.abs(g - r)
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


def field_errors(got, ref, nH, y_he=0.0, mask=None, keys=("E", "e")):
    """Per-element error of E, e and every species fraction (dict name -> error)."""
    out = {}
    for k in keys:
        out[k] = rel_error(got[k], ref[k], mask=mask)
    if "n" in ref and np.asarray(ref["n"]).size:
        fg = fractions(got["n"], nH, y_he)
        fr = fractions(ref["n"], nH, y_he)
        for k in fr:
            out[k] = rel_error(fg[k], fr[k], mask=mask)
    return out


def worst(errs):
    return max(errs.values()) if errs else 0.0
