"""Oracle of the adaptive time-step selection (Sec. 3.2.3): the local error estimate from the
explicit predictor and the next step size.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper compares the new solution U^{n+1} with the explicit predictor U^pred of the same step
(eq. explicit_predictor), weights each component by the geometric mean of the two plus one
(eq. typical_values) and takes a p-norm of the weighted difference (eq. time_error_estimator):

    w       = sqrt(|U^{n+1} U^pred|) + 1
    eps_loc = ( (1 / (N (Ns + 2))) sum |(U^{n+1} - U^pred) / w|^p )^(1/p)      (p < inf)
    eps_loc = max |(U^{n+1} - U^pred) / w|                                    (p = inf)
    dt^{n+1} = tau_tol dt^n / eps_loc                                 (eq. time_step_selection)

The weights assume normalised values; here U is the vector of Newton unknowns (e_c, n_i, E)
divided by the scalings (u_e, u_n, u_E) of Sec. 3.2.2, the same normalisation as the residual
norm.  e_c^{n+1} = e^{n+1} - e^n and the predictor's e_c is its change of e.
"""
import numpy as np

from . import model as md
from . import solve as sv


def time_error_estimate(p, U_new, U_pred, p_norm):
    """Eq. time_error_estimator with the weights of eq. typical_values on the scaled unknowns;
    p_norm = np.inf gives the max norm (no division by N (Ns + 2))."""
    u = p.scales()[:, None]
    a = np.asarray(U_new, dtype=np.float64).reshape(p.nv, p.N) / u
    b = np.asarray(U_pred, dtype=np.float64).reshape(p.nv, p.N) / u
    q = np.abs(a - b) / (np.sqrt(np.abs(a * b)) + 1.0)
    if np.isinf(p_norm):
        return float(q.max())
    return float((np.sum(q ** p_norm) / (p.N * p.nv)) ** (1.0 / p_norm))


def next_time_step(dt, eps_loc, tau_tol):
    """Eq. time_step_selection."""
    return tau_tol * dt / eps_loc


def step_with_estimate(p, state, dt, a, adot, newton_tol, p_norm, tau_tol, linear="direct"):
    """One implicit step from U^n plus its error estimate against the explicit predictor of the
    same step; returns (new_state, stats, eps_loc, dt_next)."""
    nbt = md.neighbor_table(p)
    eh = np.asarray(state["e"], dtype=np.float64).ravel()
    Un = md.state_to_U(p, state)
    T_fixed = None
    if p.isothermal:
        T_fixed = (np.asarray(state["T"], dtype=np.float64).ravel() if "T" in state
                   else md.fixed_temperature(p, state))
    U_pred = sv.explicit_predictor(p, Un, eh, dt, a, adot, T_fixed, nbt)
    new, stats = sv.implicit_step(p, state, dt, a, adot, newton_tol, linear=linear)
    eps = time_error_estimate(p, stats["U"], U_pred, p_norm)
    return new, stats, eps, next_time_step(dt, eps, tau_tol)


def ifront_radius(x_HII, dx, octants=8):
    """Radius of the ionised region of a corner source: the volume V of the cells with
    n_HII / n_H >= 1/2, mirrored into the other octants, as a sphere (Sec. 4.5)."""
    V = np.count_nonzero(np.asarray(x_HII) >= 0.5) * dx ** 3
    return (octants * 3.0 * V / (4.0 * np.pi)) ** (1.0 / 3.0)


def ifront_analytic(t, r_S, t_rec):
    """Eq. Ifront_solution: r_I = r_S (1 - exp(-t / t_rec))^(1/3)."""
    return r_S * (1.0 - np.exp(-np.asarray(t) / t_rec)) ** (1.0 / 3.0)


# --------------------------------------------------------------------------------------------
# the cosmological I-front (Sec. 4.6, "Cosmological Radiative Ionization"): a source of Ndot
# photons/s in uniform gas whose proper density falls as a^-3 in a matter-only universe of
# deceleration parameter q0.  Times are measured by the scale factor normalised to its initial
# value, a~ = a / a_i = (1 + z_i) / (1 + z); radii are comoving in units of the initial proper
# Stromgren radius r_S,i (eq. SG-stromgren_radius at z_i).

def sg_g(a, q0, z_i):
    """[1 - 2 q0 + 2 q0 (1 + z_i) / a~]^(-1/2): H0 (1 + z_i) dt = g da~ (Lambda = 0)."""
    return (1.0 - 2.0 * q0 + 2.0 * q0 * (1.0 + z_i) / np.asarray(a, dtype=np.float64)) ** -0.5


def sg_F(a, q0, z_i):
    """Eq. SG-F."""
    u = 2.0 * q0 * (1.0 + z_i) / np.asarray(a, dtype=np.float64)
    return (2.0 - 4.0 * q0 - u) * np.sqrt(1.0 - 2.0 * q0 + u)


def sg_tau(a, lam, q0, z_i):
    """Eq. SG-tau: the recombination depth lambda int_1^a~ a'^-3 g(a') da' in closed form."""
    return lam / (6.0 * q0 ** 2 * (1.0 + z_i) ** 2) * (sg_F(a, q0, z_i) - sg_F(1.0, q0, z_i))


def sg_ifront(a, lam, q0, z_i):
    """Eq. SG-solution: r_I / r_S,i at a~ >= 1, the integral of e^tau g by adaptive quadrature
    (with e^-tau(a~) taken inside it, so that a large lam does not overflow).
    lam = alpha_B n_H,i / (H0 (1 + z_i))."""
    from scipy import integrate
    out = []
    for ai in np.atleast_1d(np.asarray(a, dtype=np.float64)):
        ta = sg_tau(ai, lam, q0, z_i)
        val, _ = integrate.quad(lambda x: np.exp(sg_tau(x, lam, q0, z_i) - ta) * sg_g(x, q0, z_i),
                                1.0, ai, epsabs=0.0, epsrel=1e-12, limit=400)
        out.append((lam * val) ** (1.0 / 3.0))
    return np.asarray(out)
