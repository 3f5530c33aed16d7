"""Oracle solver: globalised Newton iteration for f(U) = 0 and one implicit time step.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The method computes the root U^{n+1} of the discrete system f(U) = 0 (eq.
nonlinear_residual) to the Newton tolerance; the Schur / CG machinery only reaches it faster.
This oracle solves the same system by a plain Newton iteration (Sec. 3.2, the quoted
algorithm below eq. nonlinear_residual) with one of three exact linear solves per step:

  "direct"        sparse LU (SuperLU) of the whole unreduced Newton matrix;
  "schur_direct"  the Schur-complement route of Sec. 3.2.1: per-cell dense solves with M
                  (step (i), eq. step_ia), the scalar system S = D - L M^-1 U solved by
                  sparse LU (step (ii)), recovery s_M = -f~_M - M^-1 U s_E (step (iii));
  "schur_cg"      as above with S solved by plain, unpreconditioned conjugate gradients to a
                  relative residual of 1e-14 (BiCGStab when the Newton matrix keeps dD/dE,
                  which makes S non-symmetric).

Readings (also listed in the design notes):
* line search (Sec. 3.2, item 2 of the Newton algorithm): a watchdog.  The full (capped) step
  is taken when it gives a new best ||f|| (by the factor 1 - 1e-4), and also when it does not,
  for at most ``watchdog`` (3) steps in a row and as long as ||f|| stays below growth_max (1e3)
  times the best; otherwise lambda is halved from 1 while ||f(U + lambda S)|| > (1 - 1e-4
  lambda) ||f(U)||, down to lam_min = 1/16 (that last step is taken).  Near bright sources the
  first Newton steps of a time step raise ||f|| before it falls quadratically: a plain Armijo
  test there accepted lambda = 1/16 steps that cut ||f|| by a few percent per iteration (18
  iterations instead of 5 on sub-boxes of the 256^3 recipe), while purely non-monotone full
  steps can cycle across the kinks of the tabulated rates;
* positivity: before the line search each cell's step is capped so that e, E and every
  species density (independent and derived) keep at least (1 - tau) of their current
  distance to their bound (fraction to the boundary, tau = 0.99); the cap multiplies the whole
  cell vector; e and E are bounded by 0, species by -1e-13 of their element total (a species
  at zero may then still move by roundoff instead of freezing its cell);
* explicit predictor (eq. explicit_predictor): the paper prints U^n + dt L^n; since L is
  defined with dU/dt = -L (eqs. mLe, mLn, mLE), the explicit Euler step is U^n - dt L(U^n);
  it is capped the same way as a Newton step.
"""
import numpy as np
from scipy import sparse
from scipy.sparse import linalg as spla

from . import closure as cl
from . import model as md


# --------------------------------------------------------------------------------------------
# bounds

def _cell_quantities(p, U, eh):
    """Quantities that must stay positive, e, E and all species (independent and derived),
    each with its roundoff allowance below zero: 0 for e and E, 1e-13 of the element total for
    the species."""
    ns = p.ns
    if ns == 0:                                    # LTE: gas and radiation energy only
        return [(eh + U[0], 0.0), (U[1], 0.0)]
    nHI, nHeI, nHeII = p.species_full(U[1:1 + ns])
    nHe = p.y_he * p.nH
    nHII, nHeIII, _ = cl.derived_species(p.nH, nHe, nHI, nHeI, nHeII)
    q = [(eh + U[0], 0.0), (U[1 + ns], 0.0), (nHI, 1e-13 * p.nH), (nHII, 1e-13 * p.nH)]
    if ns == 3:
        q += [(nHeI, 1e-13 * nHe), (nHeII, 1e-13 * nHe), (nHeIII, 1e-13 * nHe)]
    return q


def _quantity_changes(p, S):
    ns = p.ns
    if ns == 0:
        return [S[0], S[1]]
    dHI = S[1]
    out = [S[0], S[1 + ns], dHI, -dHI]
    if ns == 3:
        out += [S[2], S[3], -S[2] - S[3]]
    return out


def step_caps(p, U, eh, S):
    """Largest fraction <= 1 of the step S per cell that keeps every bounded quantity q above
    its bound -tiny by at least (1 - tau) of its current distance q + tiny (fraction to the
    boundary).  tiny = 0 for e and E; for a species it is 1e-13 of its element total, so a
    species at or near zero can still move by roundoff-sized amounts instead of freezing its
    cell."""
    cap = np.ones(p.N)
    for (q, tiny), dq in zip(_cell_quantities(p, U, eh), _quantity_changes(p, S)):
        neg = dq < 0.0
        frac = np.where(neg, p.tau * (q + tiny) / np.where(neg, -dq, 1.0), 1.0)
        cap = np.minimum(cap, np.maximum(frac, 0.0))
    return cap


# --------------------------------------------------------------------------------------------
# linear solves of J S = -f (scaled unknowns)

def cg(A, b, rtol=1e-14, maxiter=20000):
    """Plain conjugate gradients for SPD A, x0 = 0; stops at ||r||_2 <= rtol ||b||_2."""
    x = np.zeros_like(b)
    r = b.copy()
    p_ = r.copy()
    rr = r @ r
    stop = (rtol * np.sqrt(b @ b)) ** 2
    its = 0
    while rr > stop and its < maxiter:
        Ap = A @ p_
        alpha = rr / (p_ @ Ap)
        x += alpha * p_
        r -= alpha * Ap
        rr_new = r @ r
        p_ = r + (rr_new / rr) * p_
        rr = rr_new
        its += 1
    if rr > stop:
        raise RuntimeError("oracle CG did not converge")
    return x, its


def bicgstab(A, b, rtol=1e-14, maxiter=20000):
    """Plain (unpreconditioned) BiCGStab, x0 = 0; stops at ||r||_2 <= rtol ||b||_2."""
    x = np.zeros_like(b)
    r = b.copy()
    rh = r.copy()
    rho = alpha = omega = 1.0
    v = np.zeros_like(b)
    p_ = np.zeros_like(b)
    stop = rtol * np.sqrt(b @ b)
    its = 0
    while np.sqrt(r @ r) > stop and its < maxiter:
        rho_new = rh @ r
        beta = (rho_new / rho) * (alpha / omega)
        p_ = r + beta * (p_ - omega * v)
        v = A @ p_
        alpha = rho_new / (rh @ v)
        s = r - alpha * v
        its += 1
        if np.sqrt(s @ s) <= stop:
            x += alpha * p_
            r = s
            break
        t = A @ s
        omega = (t @ s) / (t @ t)
        x += alpha * p_ + omega * s
        r = s - omega * t
        rho = rho_new
    if np.sqrt(r @ r) > stop:
        raise RuntimeError("oracle BiCGStab did not converge")
    return x, its


def schur_system(p, U, f, eh, dt, a, adot, T_fixed=None, nbt=None):
    """Steps (i) and (ii) setup of Sec. 3.2.1 in scaled unknowns.

    Returns (S, rhs, fM_t, MiU): the sparse Schur matrix S = D - L M^-1 U, its right-hand
    side L f~_M - f_E, and the per-cell f~_M = M^-1 f_M and M^-1 U used in step (iii)."""
    ns, nm, N = p.ns, p.ns + 1, p.N
    nbt = md.neighbor_table(p) if nbt is None else nbt
    nb, valid = nbt
    if p.limiter_jacobian == "exact":
        return _schur_from_full_jacobian(p, U, f, eh, dt, a, adot, T_fixed, nbt)
    M, Ucol, Lrow, Dloc, lt = md.local_blocks(p, U, eh, dt, a, adot, T_fixed)
    fs = f / p.scales()[:, None]
    fM = fs[:nm].T                                           # (N, nm)
    fE = fs[nm]
    fM_t = np.linalg.solve(M, fM[:, :, None])[:, :, 0]        # step (i): M f~_M = f_M
    MiU = np.linalg.solve(M, Ucol[:, :, None])[:, :, 0]       #           M (M^-1 U) = U
    dS = Dloc - np.einsum("ij,ij->i", Lrow, MiU)
    rhs = np.einsum("ij,ij->i", Lrow, fM_t) - fE
    ddiag, drows, dcols, dvals = md.diffusion_block(p, U[nm], lt["kappa"], a, dt * p.theta, nbt)
    cells = np.arange(N)
    rows = [cells] + drows
    cols = [cells] + dcols
    vals = [dS + ddiag] + dvals
    S = sparse.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(N, N)).tocsr()
    return S, rhs, fM_t, MiU


def _schur_from_full_jacobian(p, U, f, eh, dt, a, adot, T_fixed, nbt):
    """The Schur complement by sparse block algebra on the whole Newton matrix J: with the
    local unknowns m = (e_c, n) and J_mm block diagonal (one (Ns+1)^2 block per cell),
    S = J_EE - J_Em J_mm^-1 J_mE and rhs = J_Em J_mm^-1 f_m - f_E."""
    nm, N = p.ns + 1, p.N
    J = md.full_jacobian(p, U, eh, dt, a, adot, T_fixed, nbt).tocsr()
    m_idx = np.arange(nm * N)
    E_idx = np.arange(nm * N, (nm + 1) * N)
    # per-cell blocks of J_mm (variable-major ordering: entry (r, s) of cell c at r N + c, s N + c)
    Jc = J.tocoo()
    M = np.zeros((N, nm, nm))
    sel = (Jc.row < nm * N) & (Jc.col < nm * N)
    r, s = Jc.row[sel], Jc.col[sel]
    assert np.all(r % N == s % N), "J_mm is not block diagonal"
    np.add.at(M, (r % N, r // N, s // N), Jc.data[sel])
    JmE = J[m_idx][:, E_idx].tocoo()
    Ucol = np.zeros((N, nm))
    assert np.all(JmE.row % N == JmE.col), "J_mE is not cell-local"
    np.add.at(Ucol, (JmE.col, JmE.row // N), JmE.data)
    fs = f / p.scales()[:, None]
    fM_t = np.linalg.solve(M, fs[:nm].T[:, :, None])[:, :, 0]
    MiU = np.linalg.solve(M, Ucol[:, :, None])[:, :, 0]
    cells = np.arange(N)
    MiU_mat = sparse.coo_matrix((MiU.T.ravel(), (np.repeat(np.arange(nm), N) * N + np.tile(cells, nm),
                                                 np.tile(cells, nm))), shape=(nm * N, N)).tocsr()
    JEm = J[E_idx][:, m_idx]
    JEE = J[E_idx][:, E_idx]
    S = (JEE - JEm @ MiU_mat).tocsr()
    rhs = JEm @ fM_t.T.ravel() - fs[nm]
    return S, rhs, fM_t, MiU


def newton_direction(p, U, f, eh, dt, a, adot, T_fixed=None, nbt=None, linear="direct"):
    """Solve J(U) S = -f(U) exactly (up to roundoff); returns the physical step S (nv, N)
    and the number of inner iterations (0 for direct solves)."""
    u = p.scales()[:, None]
    nm = p.ns + 1
    if linear == "direct":
        J = md.full_jacobian(p, U, eh, dt, a, adot, T_fixed, nbt)
        fs = (f / u).ravel()
        s = spla.spsolve(J.tocsc(), -fs).reshape(p.nv, p.N)
        return s * u, 0
    S, rhs, fM_t, MiU = schur_system(p, U, f, eh, dt, a, adot, T_fixed, nbt)
    if linear == "schur_direct":
        sE = spla.spsolve(S.tocsc(), rhs)
        its = 0
    elif linear == "schur_cg":
        sE, its = cg(S, rhs) if p.limiter_jacobian == "lagged" else bicgstab(S, rhs)
    else:
        raise ValueError(linear)
    sM = -fM_t - MiU * sE[:, None]                             # step (iii)
    s = np.empty((p.nv, p.N))
    s[:nm] = sM.T
    s[nm] = sE
    return s * u, its


# --------------------------------------------------------------------------------------------
# the Newton iteration and one implicit step

def newton(p, U0, g, eh, dt, a, adot, tol, T_fixed=None, linear="direct", max_newton=50):
    """Globalised inexact Newton iteration (Sec. 3.2) from U0 until ||f||_RMS < tol."""
    nbt = md.neighbor_table(p)
    U = U0.copy()
    f = md.residual(p, U, g, eh, dt, a, adot, T_fixed, nbt)
    r = md.rms_norm(p, f)
    stats = dict(newton_its=0, linear_its=0, backtracks=0, full_step_fallbacks=0,
                 res_history=[r], converged=False)
    r_best, bad = r, 0
    for _ in range(max_newton):
        if r < tol:
            break
        S, its = newton_direction(p, U, f, eh, dt, a, adot, T_fixed, nbt, linear)
        stats["linear_its"] += its
        cap = step_caps(p, U, eh, S)

        def trial(lam):
            Ut = U + np.minimum(lam, cap)[None, :] * S
            ft = md.residual(p, Ut, g, eh, dt, a, adot, T_fixed, nbt)
            return Ut, ft, md.rms_norm(p, ft)

        Ut, ft, rt = trial(1.0)
        if rt <= (1.0 - 1e-4) * r_best:            # a new best residual
            r_best, bad = rt, 0
        elif bad < p.watchdog and rt <= p.growth_max * r_best:
            bad += 1                               # tolerated non-monotone full step
        else:                                      # Armijo backtracking from U
            lam = 1.0
            while not rt <= (1.0 - 1e-4 * lam) * r:
                if lam * 0.5 < p.lam_min:
                    stats["full_step_fallbacks"] += 1
                    break
                lam *= 0.5
                stats["backtracks"] += 1
                Ut, ft, rt = trial(lam)
            bad = 0
            r_best = min(r_best, rt)
        U, f, r = Ut, ft, rt
        stats["newton_its"] += 1
        stats["res_history"].append(r)
    stats["converged"] = bool(r < tol)
    stats["residual"] = r
    return U, stats


def explicit_predictor(p, Un, eh, dt, a, adot, T_fixed=None, nbt=None):
    """Eq. explicit_predictor, read as the explicit Euler step U^n - dt L(U^n), capped."""
    d = -dt * md.full_operator(p, Un, eh, a, adot, T_fixed, nbt)
    cap = step_caps(p, Un, eh, d)
    return Un + cap[None, :] * d


def implicit_step(p, state, dt, a, adot, newton_tol, guess="prev", U0=None, linear="direct",
                  max_newton=50):
    """One step t^n -> t^{n+1} of eqs. RT-cons_energy .. RT-cons_radiation (theta scheme).

    state: dict with E (N,), e (N,) (specific gas energy e^n = e_h), n (ns, N); isothermal
    runs hold the temperature state["T"] (default: the temperature of the given state) and
    carry it into the returned state.
    guess: "prev" (U^n), "predictor" (eq. explicit_predictor) or "given" (U0).
    Returns (new_state, stats); e^{n+1} = e_h + e_c (Sec. 3.1 with no hydrodynamics)."""
    nbt = md.neighbor_table(p)
    eh = np.asarray(state["e"], dtype=np.float64).ravel()
    Un = md.state_to_U(p, state)
    T_fixed = None
    if p.isothermal:        # the temperature of the state first handed in is held fixed
        T_fixed = (np.asarray(state["T"], dtype=np.float64).ravel() if "T" in state
                   else md.fixed_temperature(p, state))
    g = md.build_g(p, Un, eh, dt, a, adot, T_fixed, nbt)
    if guess == "prev":
        start = Un
    elif guess == "predictor":
        start = explicit_predictor(p, Un, eh, dt, a, adot, T_fixed, nbt)
    elif guess == "given":
        start = np.asarray(U0, dtype=np.float64).reshape(p.nv, p.N)
    else:
        raise ValueError(guess)
    U, stats = newton(p, start, g, eh, dt, a, adot, newton_tol, T_fixed, linear, max_newton)
    ns = p.ns
    new = dict(E=U[1 + ns].copy(), e=eh + U[0], n=U[1:1 + ns].copy())
    if p.isothermal:
        new["T"] = T_fixed
    stats["U"] = U
    return new, stats
