"""Oracle closure: constants, rate/cooling table, equation of state, grey spectral constants.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper prints the structure of the coupling terms but not their formulas: the ionisation,
recombination, heating and cooling rates are only cited (Sec. 2.1, "Model Coupling", nLTE
case).  The closure below is therefore a project definition, written in the functional forms
of the published fits the paper cites for these coefficients:

* case-B radiative recombination of HII / HeII / HeIII and case-B recombination cooling in
  the forms of Hui & Gnedin (1997) (cited by the paper for the rate coefficients, Sec. 2);
  the HII rate reproduces the value alpha_B(1e4 K) = 2.59e-13 cm^3/s printed in Sec. 4.5;
* collisional ionisation, collisional-ionisation / collisional-excitation cooling,
  dielectronic recombination and bremsstrahlung in the forms of Cen (1992) and Black (1981)
  (both cited in Sec. 2.1).

As in Enzo (the code the paper is built in), the temperature-dependent coefficients are
tabulated once and linearly interpolated inside the solve.  The table nodes sit on a grid that
is exact in binary: 2^TABLE_BITS bins per octave of T over [1 K, 2^30 K).  A temperature's bin
is its binary exponent plus the top TABLE_BITS bits of its mantissa, so the bin choice is exact
and identical on every platform.  Outside the table range T is clamped and its derivative is 0.
"""
import math

import numpy as np
from scipy import integrate

# --------------------------------------------------------------------------------------------
# CGS constants
C_LIGHT = 2.99792458e10          # cm / s
K_BOLTZ = 1.380649e-16           # erg / K
M_H = 1.67262192e-24             # g, the proton mass m_p of eq. temperature
EV = 1.602176634e-12             # erg
H_PLANCK = 6.62607015e-27        # erg s
GAMMA = 5.0 / 3.0                # ratio of specific heats (Sec. 2, below eq. eos)
SIGMA_SB = 5.670374419e-5        # erg cm^-2 s^-1 K^-4, Stefan-Boltzmann constant (eq. LTE_coupling)
A_RAD = 4.0 * SIGMA_SB / C_LIGHT # erg cm^-3 K^-4, radiation constant

# ionisation thresholds (hnu_0 = 13.6 eV for hydrogen, Sec. 2.2)
E_THR = np.array([13.6 * EV, 24.6 * EV, 54.4 * EV])        # HI, HeI, HeII
# threshold photoionisation cross sections, cm^2 (6.3e-18 for HI as in the configs)
SIGMA_THR = np.array([6.30e-18, 7.42e-18, 1.575e-18])

# threshold temperatures chi / k_B used inside the Hui & Gnedin fits
T_HI, T_HEI, T_HEII = 157807.0, 285335.0, 631515.0

# --------------------------------------------------------------------------------------------
# rate / cooling coefficients (column order of the table)
RATE_NAMES = (
    "alpha_HII",    # HII  + e -> HI          (case B)              cm^3/s
    "beta_HI",      # HI   + e -> HII + 2e    (collisional ion.)    cm^3/s
    "alpha_HeII",   # HeII + e -> HeI         (case B + dielectronic)
    "beta_HeI",     # HeI  + e -> HeII + 2e
    "alpha_HeIII",  # HeIII+ e -> HeII        (case B)
    "beta_HeII",    # HeII + e -> HeIII + 2e
    "cool_HI",      # cooling coefficient multiplying n_e n_HI     erg cm^3/s
    "cool_HII",     # ... n_e n_HII
    "cool_HeI",     # ... n_e n_HeI
    "cool_HeII",    # ... n_e n_HeII
    "cool_HeIII",   # ... n_e n_HeIII
)
NRATES = len(RATE_NAMES)


def _hg97_caseB_rate(T, T_thr):
    """Hui & Gnedin (1997) case-B recombination rate of a hydrogen-like ion, cm^3/s."""
    lam = 2.0 * T_thr / T
    return 2.753e-14 * lam ** 1.5 / (1.0 + (lam / 2.740) ** 0.407) ** 2.242


def _hg97_caseB_cool(T, T_thr):
    """Hui & Gnedin (1997) case-B recombination cooling of a hydrogen-like ion, erg cm^3/s."""
    lam = 2.0 * T_thr / T
    return 3.435e-30 * T * lam ** 1.970 / (1.0 + (lam / 2.250) ** 0.376) ** 3.720


def _hg97_HeII_caseB_rate(T):
    """Hui & Gnedin (1997) case-B radiative recombination HeII -> HeI, cm^3/s."""
    return 1.26e-14 * (2.0 * T_HEI / T) ** 0.75


def _dielectronic_rate(T):
    """Dielectronic recombination HeII -> HeI (Cen 1992 form), cm^3/s."""
    return 1.90e-3 * T ** -1.5 * np.exp(-470000.0 / T) * (1.0 + 0.3 * np.exp(-94000.0 / T))


def _gaunt(T):
    """Free-free Gaunt factor of the Cen (1992) bremsstrahlung fit."""
    return 1.1 + 0.34 * np.exp(-(5.5 - np.log10(T)) ** 2 / 3.0)


def closure_terms(T):
    """Every named term of the closure at temperature(s) T (K), as a dict of arrays."""
    T = np.asarray(T, dtype=np.float64)
    sq = np.sqrt(T)
    d5 = 1.0 + np.sqrt(T / 1e5)
    t = {}
    t["alpha_HII_B"] = _hg97_caseB_rate(T, T_HI)
    t["alpha_HeII_B"] = _hg97_HeII_caseB_rate(T)
    t["alpha_HeII_di"] = _dielectronic_rate(T)
    t["alpha_HeIII_B"] = 2.0 * _hg97_caseB_rate(T, T_HEII)
    t["beta_HI"] = 5.85e-11 * sq * np.exp(-157809.1 / T) / d5
    t["beta_HeI"] = 2.38e-11 * sq * np.exp(-285335.4 / T) / d5
    t["beta_HeII"] = 5.68e-12 * sq * np.exp(-631515.0 / T) / d5
    t["cool_ci_HI"] = 1.27e-21 * sq * np.exp(-157809.1 / T) / d5
    t["cool_ci_HeI"] = 9.38e-22 * sq * np.exp(-285335.4 / T) / d5
    t["cool_ci_HeII"] = 4.95e-22 * sq * np.exp(-631515.0 / T) / d5
    t["cool_ce_HI"] = 7.50e-19 * np.exp(-118348.0 / T) / d5
    t["cool_ce_HeII"] = 5.54e-17 * T ** -0.397 * np.exp(-473638.0 / T) / d5
    t["cool_rec_HII"] = _hg97_caseB_cool(T, T_HI)
    t["cool_rec_HeII"] = K_BOLTZ * T * _hg97_HeII_caseB_rate(T)
    t["cool_rec_HeIII"] = 8.0 * _hg97_caseB_cool(T, T_HEII)
    t["cool_di_HeII"] = (1.24e-13 * T ** -1.5 * np.exp(-470000.0 / T)
                         * (1.0 + 0.3 * np.exp(-94000.0 / T)))
    t["brem"] = 1.42e-27 * _gaunt(T) * sq       # times Z^2 n_e n_ion
    return t


def rate_formulas(T):
    """All closure coefficients at temperature(s) T (K), shape T.shape + (NRATES,).

    These are the smooth formulas the table is built from.  Tests also use them directly as
    a smooth closure (e.g. for finite-difference Jacobian checks)."""
    t = closure_terms(T)
    out = np.empty(np.shape(T) + (NRATES,))
    out[..., 0] = t["alpha_HII_B"]
    out[..., 1] = t["beta_HI"]
    out[..., 2] = t["alpha_HeII_B"] + t["alpha_HeII_di"]
    out[..., 3] = t["beta_HeI"]
    out[..., 4] = t["alpha_HeIII_B"]
    out[..., 5] = t["beta_HeII"]
    out[..., 6] = t["cool_ce_HI"] + t["cool_ci_HI"]
    out[..., 7] = t["cool_rec_HII"] + t["brem"]
    out[..., 8] = t["cool_ci_HeI"]
    out[..., 9] = (t["cool_ci_HeII"] + t["cool_ce_HeII"] + t["cool_rec_HeII"]
                   + t["cool_di_HeII"] + t["brem"])
    out[..., 10] = t["cool_rec_HeIII"] + 4.0 * t["brem"]
    return out


# --------------------------------------------------------------------------------------------
# the table
TABLE_BITS = 6                       # 64 bins per octave
TABLE_OCTAVES = 30                   # T in [2^0, 2^30) K
NBINS = TABLE_OCTAVES << TABLE_BITS
T_TABLE_MIN = 1.0
T_TABLE_MAX = math.nextafter(2.0 ** TABLE_OCTAVES, 0.0)


def table_nodes():
    """Node temperatures T_i = 2^(i // 64) * (1 + (i % 64) / 64), i = 0..NBINS (inclusive)."""
    i = np.arange(NBINS + 1)
    octave = i >> TABLE_BITS
    j = i & ((1 << TABLE_BITS) - 1)
    return np.ldexp(1.0 + j / float(1 << TABLE_BITS), octave)


class RateTable:
    """Piecewise-linear interpolant of ``rate_formulas`` on the binary node grid.

    value(T) = k_i + s_i (T - T_i) in bin i, s_i = (k_{i+1} - k_i) / (T_{i+1} - T_i)."""

    def __init__(self, formulas=rate_formulas):
        self.T = table_nodes()
        self.k = formulas(self.T)                                       # (NBINS+1, NRATES)
        self.s = (self.k[1:] - self.k[:-1]) / (self.T[1:] - self.T[:-1])[:, None]

    @staticmethod
    def bin_of(Tc):
        """Bin index of clamped temperatures: binary exponent and top mantissa bits."""
        m, ex = np.frexp(Tc)                   # Tc = m 2^ex, m in [0.5, 1)
        frac = 2.0 * m - 1.0                   # exact
        j = np.floor(frac * (1 << TABLE_BITS)).astype(np.int64)
        return ((ex.astype(np.int64) - 1) << TABLE_BITS) + j

    def __call__(self, T):
        """Returns (k, dk/dT) with shape T.shape + (NRATES,); dk/dT = 0 where T is clamped."""
        T = np.asarray(T, dtype=np.float64)
        Tc = np.clip(T, T_TABLE_MIN, T_TABLE_MAX)
        clamped = (T < T_TABLE_MIN) | (T > T_TABLE_MAX)
        b = self.bin_of(Tc)
        s = self.s[b]
        k = self.k[b] + s * (Tc - self.T[b])[..., None]
        dk = np.where(clamped[..., None], 0.0, s)
        return k, dk


class SmoothRates:
    """The closure formulas themselves with a centred-difference derivative (tests only)."""

    def __call__(self, T):
        T = np.asarray(T, dtype=np.float64)
        h = 1e-6 * T
        k = rate_formulas(T)
        dk = (rate_formulas(T + h) - rate_formulas(T - h)) / (2.0 * h)[..., None]
        return k, dk


# --------------------------------------------------------------------------------------------
# equation of state and species bookkeeping (Sec. 2, eqs. eos and temperature)

def derived_species(nH, nHe, nHI, nHeI, nHeII):
    """n_HII, n_HeIII and n_e from the independent species (element conservation)."""
    nHII = nH - nHI
    nHeIII = nHe - nHeI - nHeII
    ne = nHII + nHeII + 2.0 * nHeIII
    return nHII, nHeIII, ne


def mass_density(nH, nHe):
    """rho_b = m_H (n_H + 4 n_He)."""
    return M_H * (nH + 4.0 * nHe)


def temperature(e, nH, nHe, ne):
    """Eq. temperature with eq. eos at v_b = 0: p = (gamma-1) rho e, T = p / (n_tot k_B)."""
    ntot = nH + nHe + ne
    return (GAMMA - 1.0) * mass_density(nH, nHe) * e / (K_BOLTZ * ntot)


# --------------------------------------------------------------------------------------------
# grey spectral constants (Sec. 2.2 eq. grey_definition; Sec. 3.2.5 eq. adaptive_spectrum)

def _cross_section_ratio(nu_ratio):
    """sigma(nu) / sigma(nu_X) = (nu / nu_X)^-3 above threshold (hydrogenic form)."""
    return nu_ratio ** -3.0


def grey_constants(kind, param=None, nspecies=3):
    """Frequency-integrated constants of the grey equations, per absorber HI, HeI, HeII.

    kind = "mono": radiation at a single photon energy ``param`` (erg); chi = delta.
    kind = "blackbody": chi(nu) ~ nu^3 / (exp(h nu / k T_B) - 1), param = T_B (K).
    kind = "powerlaw": chi(nu) = (nu / nu_0)^alpha, alpha = param < -1.

    Returns a dict of arrays over absorbers:
      sk   = int sigma chi dnu / int chi dnu                 (cm^2, opacity per absorber)
      pgam = int sigma chi / (h nu) dnu / int chi dnu        (cm^2/erg, Gamma = c pgam E)
      ph   = int sigma chi (1 - nu_X/nu) dnu / int chi dnu   (cm^2, heating G = c ph n E)
      eps  = int chi dnu / int chi / (h nu) dnu              (erg, mean photon energy)
    Integrals run from the hydrogen threshold nu_0 to infinity (eq. grey_definition).
    Absorbers beyond ``nspecies`` (H-only runs) are zero."""
    sk = np.zeros(3)
    pgam = np.zeros(3)
    ph = np.zeros(3)
    if kind == "mono":
        hnu = float(param)
        for X in range(nspecies):
            if hnu >= E_THR[X]:
                sig = SIGMA_THR[X] * _cross_section_ratio(hnu / E_THR[X])
                sk[X] = sig
                pgam[X] = sig / hnu
                ph[X] = sig * (1.0 - E_THR[X] / hnu)
        return dict(sk=sk, pgam=pgam, ph=ph, eps=hnu)

    # integrate in x = h nu / E_0 (E_0 = 13.6 eV); chi is only needed up to a constant
    E0 = E_THR[0]
    if kind == "blackbody":
        kT = K_BOLTZ * float(param)

        def chi(x):
            y = x * E0 / kT
            return x ** 3 / math.expm1(y) if y < 700.0 else 0.0
    elif kind == "powerlaw":
        alpha = float(param)
        if not alpha < -1.0:
            raise ValueError("power-law index must be < -1")

        def chi(x):
            return x ** alpha
    else:
        raise ValueError(kind)

    def quad(f, lo):
        val, err = integrate.quad(f, lo, np.inf, epsabs=0.0, epsrel=1e-13, limit=400)
        return val

    Z = quad(chi, 1.0)
    Zphot = quad(lambda x: chi(x) / (x * E0), 1.0)
    for X in range(nspecies):
        xX = E_THR[X] / E0
        sig = lambda x, xX=xX, X=X: SIGMA_THR[X] * _cross_section_ratio(x / xX)
        sk[X] = quad(lambda x: sig(x) * chi(x), xX) / Z
        pgam[X] = quad(lambda x: sig(x) * chi(x) / (x * E0), xX) / Z
        ph[X] = quad(lambda x: sig(x) * chi(x) * (1.0 - xX / x), xX) / Z
    return dict(sk=sk, pgam=pgam, ph=ph, eps=Z / Zphot)


def deposit_sources(shape, dx, ijk, photons_per_s, eps):
    """Emissivity field 4 pi eta (erg cm^-3 s^-1, comoving): each point source puts
    Ndot * eps into its cell's comoving volume dx^3.  ``ijk`` rows are (i, j, k); array
    layout is [k, j, i] (x fastest)."""
    src = np.zeros(shape)
    vol = dx ** 3
    for (i, j, k), nd in zip(np.asarray(ijk).reshape(-1, 3), np.asarray(photons_per_s).ravel()):
        src[k, j, i] += nd * eps / vol
    return src
