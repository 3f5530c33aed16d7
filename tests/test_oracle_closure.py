"""Pins of the oracle closure against values the paper prints and against closed forms."""
import math
import os

import numpy as np
import pytest
from scipy import special

from oracle import closure as cl
from paper_0901_1110_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KPC = 3.0857e21


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            key, val = line.split()[:2]
            vals[key] = float(val)
    return vals


def test_caseB_recombination_matches_printed_value():
    """Sec. 4.5 prints alpha_B = 2.59e-13 cm^3/s for the T = 1e4 K test."""
    g = _golden("iliev_test1_paper_values.txt")
    a_formula = cl.closure_terms(np.array([g["T"]]))["alpha_HII_B"][0]
    a_table = cl.RateTable()(np.array([g["T"]]))[0][0, 0]
    assert abs(a_formula / g["alpha_B"] - 1) < 5e-3
    assert abs(a_table / g["alpha_B"] - 1) < 5e-3


def test_stromgren_radius_and_recombination_time_match_paper():
    """Eq. Stromgren_radius and t_rec = 1/(alpha_B n_H) with the closure's alpha_B reproduce
    the printed r_S = 5.4 kpc and t_rec = 3.86e15 s (Sec. 4.5)."""
    g = _golden("iliev_test1_paper_values.txt")
    alpha = cl.closure_terms(np.array([g["T"]]))["alpha_HII_B"][0]
    rS = (3.0 * g["Ndot_gamma"] / (4.0 * math.pi * alpha * g["n_H"] ** 2)) ** (1.0 / 3.0)
    assert abs(rS / KPC - g["r_S"]) < 0.05
    trec = 1.0 / (alpha * g["n_H"])
    assert abs(trec / g["t_rec"] - 1) < 5e-3


@pytest.mark.parametrize("T", [8e3, 2e4, 1e5, 1e6])
def test_collisional_ionisation_cooling_is_threshold_energy_times_rate(T):
    """Each collisional ionisation removes the ionisation energy (13.6, 24.6, 54.4 eV): the
    cooling fits divided by the rate fits must give those energies (catches a mistyped
    constant in either)."""
    t = cl.closure_terms(np.array([T]))
    for cool, rate, chi in (("cool_ci_HI", "beta_HI", 13.6), ("cool_ci_HeI", "beta_HeI", 24.6),
                            ("cool_ci_HeII", "beta_HeII", 54.4)):
        assert abs(t[cool][0] / t[rate][0] / cl.EV / chi - 1) < 5e-3


def test_hydrogenic_scaling_of_HeIII_recombination():
    """alpha(Z=2, T) = Z alpha_H(T / Z^2) for a hydrogen-like ion (thresholds 4:1)."""
    T = np.array([3e3, 1e4, 1e5])
    t = cl.closure_terms(T)
    tH = cl.closure_terms(T * cl.T_HI / cl.T_HEII)
    np.testing.assert_allclose(t["alpha_HeIII_B"], 2.0 * tH["alpha_HII_B"], rtol=1e-12)


def test_recombination_cooling_energy_is_a_fraction_of_kT():
    """Case-B recombination cooling per recombination lies between 0.5 and 1 k_B T at
    1e3..3e4 K (hydrogen recombination removes a thermal-energy fraction below kT)."""
    T = np.array([1e3, 1e4, 3e4])
    t = cl.closure_terms(T)
    ratio = t["cool_rec_HII"] / (cl.K_BOLTZ * T * t["alpha_HII_B"])
    assert np.all((ratio > 0.5) & (ratio < 1.0))


def test_table_nodes_exact_and_bins_match_search():
    tab = cl.RateTable()
    np.testing.assert_array_equal(tab.k, cl.rate_formulas(tab.T))
    rng = np.random.default_rng(0)
    T = np.exp(rng.uniform(0.0, math.log(2.0 ** 30) - 1e-9, 20000))
    b = cl.RateTable.bin_of(T)
    ref = np.searchsorted(tab.T, T, side="right") - 1
    np.testing.assert_array_equal(b, ref)
    # node temperatures themselves fall in their own bin
    np.testing.assert_array_equal(cl.RateTable.bin_of(tab.T[:-1]), np.arange(cl.NBINS))


def test_table_is_the_piecewise_linear_interpolant():
    tab = cl.RateTable()
    i = np.arange(0, cl.NBINS, 37)
    mid = 0.5 * (tab.T[i] + tab.T[i + 1])
    k, dk = tab(mid)
    np.testing.assert_allclose(k, 0.5 * (tab.k[i] + tab.k[i + 1]), rtol=1e-13, atol=1e-300)
    np.testing.assert_allclose(dk, (tab.k[i + 1] - tab.k[i]) / (tab.T[i + 1] - tab.T[i])[:, None],
                               rtol=1e-13, atol=1e-300)
    # clamped below the table: value at 1 K, zero derivative
    k0, dk0 = tab(np.array([0.25]))
    np.testing.assert_allclose(k0[0], tab.k[0], rtol=1e-15)
    assert np.all(dk0 == 0.0)
    # the table tracks the smooth formulas (64 bins per octave) wherever a coefficient is
    # not negligible; exponentially small values (e.g. exp(-470000/T) at 50 K) are not tracked
    T = np.geomspace(50.0, 1e8, 301)
    ref = cl.rate_formulas(T)
    big = ref >= 1e-8 * ref.max(axis=0)
    rel = np.abs(tab(T)[0] - ref) / np.where(big, ref, 1.0)
    assert rel[big].max() < 5e-2
    assert np.median(rel[big]) < 1e-4


def _bose_moment(n, y0, kmax=400):
    """int_{y0}^inf y^n / (e^y - 1) dy for n = 2, 3 by its exponential series."""
    k = np.arange(1, kmax + 1)
    e = np.exp(-k * y0)
    if n == 3:
        return float(np.sum(e * (y0 ** 3 / k + 3 * y0 ** 2 / k ** 2 + 6 * y0 / k ** 3 + 6 / k ** 4)))
    if n == 2:
        return float(np.sum(e * (y0 ** 2 / k + 2 * y0 / k ** 2 + 2 / k ** 3)))
    raise ValueError


@pytest.mark.parametrize("TB", [3e4, 1e5, 3e5])
def test_blackbody_grey_constants_closed_form(TB):
    """Eq. adaptive_spectrum for a T_B blackbody (Sec. 2.2) with sigma ~ nu^-3: the
    frequency integrals have closed forms in the Bose series, -ln(1 - e^-y) and E_1."""
    g = cl.grey_constants("blackbody", TB, 3)
    kT = cl.K_BOLTZ * TB
    y0 = cl.E_THR[0] / kT
    Z3 = _bose_moment(3, y0)
    Z2 = _bose_moment(2, y0)
    assert abs(g["eps"] / (kT * Z3 / Z2) - 1) < 1e-10
    k = np.arange(1, 400)
    for X in range(3):
        yX = cl.E_THR[X] / kT
        pref = cl.SIGMA_THR[X] * yX ** 3 / Z3
        I0 = -math.log1p(-math.exp(-yX))                      # int dy / (e^y - 1)
        Im1 = float(np.sum(special.exp1(k * yX)))               # int dy / (y (e^y - 1))
        assert abs(g["sk"][X] / (pref * I0) - 1) < 1e-10
        assert abs(g["pgam"][X] / (pref * Im1 / kT) - 1) < 1e-10
        assert abs(g["ph"][X] / (pref * (I0 - yX * Im1)) - 1) < 1e-9


@pytest.mark.parametrize("alpha", [-1.5, -3.0])
def test_powerlaw_grey_constants_closed_form(alpha):
    g = cl.grey_constants("powerlaw", alpha, 3)
    E0 = cl.E_THR[0]
    assert abs(g["eps"] / (E0 * (-alpha) / (-alpha - 1)) - 1) < 1e-11
    for X in range(3):
        tX = cl.E_THR[X] / E0
        sk = cl.SIGMA_THR[X] * tX ** (alpha + 1) * (-alpha - 1) / (2 - alpha)
        pg = cl.SIGMA_THR[X] * tX ** alpha * (-alpha - 1) / ((3 - alpha) * E0)
        assert abs(g["sk"][X] / sk - 1) < 1e-11
        assert abs(g["pgam"][X] / pg - 1) < 1e-11
        assert abs(g["ph"][X] / (sk - cl.E_THR[X] * pg) - 1) < 1e-9


def test_monochromatic_threshold_constants():
    """Monochromatic 13.6 eV radiation (the 32^3 benchmark): no heating, no helium
    photoionisation, Gamma = c sigma E / h nu."""
    g = cl.grey_constants("mono", 13.6 * cl.EV, 3)
    assert g["sk"][0] == 6.3e-18 and g["ph"][0] == 0.0
    assert g["pgam"][0] == 6.3e-18 / (13.6 * cl.EV)
    assert np.all(g["sk"][1:] == 0.0) and np.all(g["pgam"][1:] == 0.0)


def test_generator_initial_energy_gives_the_requested_temperature():
    """The workload's initial e (from T0) maps back to T0 through eqs. eos / temperature."""
    for w in (inputs.uniform_h(6), inputs.lognormal_hhe((5, 6, 7), nsrc=2)):
        n = w.n.reshape(w.ns, -1)
        nH = w.nH.ravel()
        nHe = w.y_he * nH
        z = np.zeros_like(nH)
        nHI, nHeI, nHeII = (n[0], z, z) if w.ns == 1 else (n[0], n[1], n[2])
        _, _, ne = cl.derived_species(nH, nHe, nHI, nHeI, nHeII)
        T = cl.temperature(w.e.ravel(), nH, nHe, ne)
        np.testing.assert_allclose(T, 100.0, rtol=1e-13)


def test_source_deposit_conserves_photon_energy_rate():
    ijk = np.array([[1, 2, 3], [1, 2, 3], [0, 0, 0]])
    rate = np.array([1e48, 2e48, 5e47])
    src = cl.deposit_sources((4, 5, 6), 2.0, ijk, rate, 3.0)
    assert abs(src.sum() * 8.0 - rate.sum() * 3.0) < 1e-12 * rate.sum() * 3.0
    assert src[3, 2, 1] == 3e48 * 3.0 / 8.0


# ---- the terms of the closure whose constants no printed value fixes: pins from physics that
# the code does not contain (fundamental constants, transition energies, detailed balance of
# collisional excitation)

# CGS fundamental constants used only by these pins
E_CHARGE = 4.80320471e-10        # esu
M_E = 9.1093837015e-28           # g


def test_bremsstrahlung_prefactor_from_fundamental_constants():
    """Free-free emission of a thermal plasma (Rybicki & Lightman 1979, eq. 5.15b):
    eps_ff = (2^5 pi e^6 / (3 h m_e c^3)) (2 pi k T / (3 m_e))^(1/2) Z^2 n_e n_i g_B.  The
    closure's amplitude divided by its Gaunt factor and sqrt(T) equals that prefactor (1.4256e-27
    cgs) to the three figures the fit quotes."""
    pref = (2 ** 5 * math.pi * E_CHARGE ** 6 / (3 * cl.H_PLANCK * M_E * cl.C_LIGHT ** 3)
            * math.sqrt(2 * math.pi * cl.K_BOLTZ / (3 * M_E)))
    T = np.logspace(3, 8, 11)
    t = cl.closure_terms(T)
    amp = t["brem"] / (np.sqrt(T) * cl._gaunt(T))
    np.testing.assert_allclose(amp, pref, rtol=5e-3)


def test_bremsstrahlung_gaunt_factor_in_its_physical_range():
    """The frequency-averaged free-free Gaunt factor lies between 1.1 and 1.5 (Rybicki &
    Lightman 1979, Sec. 5.2); the fit peaks at log10 T = 5.5."""
    T = np.logspace(2, 9, 71)
    g = cl._gaunt(T)
    assert np.all((g >= 1.1) & (g <= 1.5))
    assert abs(np.log10(T[np.argmax(g)]) - 5.5) < 0.05


def test_collisional_excitation_thresholds_are_the_lyman_alpha_energies():
    """Collisional excitation of HI and HeII cools through the n = 1 -> 2 transition of a
    hydrogen-like ion, 3/4 of its ionisation energy (10.2 eV and 40.8 eV): the temperature in
    the Boltzmann factor of each fit, recovered from the fit at T and 2T with the fit's other
    T-dependence divided out, is that energy over k_B."""
    T = np.array([2e4, 1e5, 4e5])
    d5 = lambda x: 1.0 + np.sqrt(x / 1e5)
    for key, chi, pw in (("cool_ce_HI", 13.6, 0.0), ("cool_ce_HeII", 54.4, -0.397)):
        t1 = cl.closure_terms(T)[key]
        t2 = cl.closure_terms(2 * T)[key]
        boltz_ratio = (t2 / t1) * (d5(2 * T) / d5(T)) / 2.0 ** pw
        T_exp = np.log(boltz_ratio) / (1.0 / T - 1.0 / (2 * T))
        np.testing.assert_allclose(T_exp, 0.75 * chi * cl.EV / cl.K_BOLTZ, rtol=1e-3)


def _collision_strength(cool, T, dE, g1=2.0):
    """Effective collision strength of a collisional-excitation cooling coefficient
    cool = dE q12 with q12 = 8.629e-6 Omega / (g1 sqrt(T)) exp(-dE / kT) cm^3/s (detailed
    balance of collisional excitation, Osterbrock & Ferland 2006, Sec. 3.5)."""
    return cool * np.sqrt(T) * g1 / (8.629e-6 * dE * np.exp(-dE / (cl.K_BOLTZ * T)))


def test_collisional_excitation_amplitudes_give_physical_collision_strengths():
    """The HI and HeII excitation cooling fits correspond to effective collision strengths of
    order one for HI (0.3..3 over 5e3..1e5 K) and about 1/Z^2 of that for HeII; hydrogenic
    scaling Z^2 Omega_HeII(Z^2 T) ~ Omega_HI(T) holds within the spread of the fits.  A slip
    of a decade in either amplitude fails."""
    T = np.array([5e3, 1e4, 2e4, 5e4, 1e5])
    dH, dHe = 0.75 * 13.6 * cl.EV, 0.75 * 54.4 * cl.EV
    oH = _collision_strength(cl.closure_terms(T)["cool_ce_HI"], T, dH)
    oHe = _collision_strength(cl.closure_terms(4 * T)["cool_ce_HeII"], 4 * T, dHe)
    assert np.all((oH > 0.3) & (oH < 3.0)), oH
    assert np.all((oHe > 0.1) & (oHe < 1.0)), oHe
    r = 4.0 * oHe / oH
    assert np.all((r > 0.4) & (r < 2.5)), r


def test_dielectronic_recombination_cools_by_the_core_transition_energy():
    """Dielectronic recombination of HeII proceeds through the 1s -> 2p excitation of the core
    (40.8 eV): each recombination carries that energy away (the cooling fit over the rate fit),
    and the Boltzmann factor of the resonance uses it (exponent temperature within 1%)."""
    T = np.logspace(4, 7, 7)
    t = cl.closure_terms(T)
    per = t["cool_di_HeII"] / t["alpha_HeII_di"] / cl.EV
    np.testing.assert_allclose(per, 40.8, rtol=5e-3)
    dE = 0.75 * 54.4 * cl.EV
    # d ln(alpha T^1.5) / d(1/T) = -T0 (1 + small second resonance term)
    Tb = np.array([3e4, 4e4])
    a = cl.closure_terms(Tb)["alpha_HeII_di"] * Tb ** 1.5
    T0 = -np.log(a[1] / a[0]) / (1.0 / Tb[1] - 1.0 / Tb[0])
    assert abs(T0 / (dE / cl.K_BOLTZ) - 1.0) < 1e-2, T0


def test_helium_case_b_recombination_close_to_hydrogen_at_nebular_temperatures():
    """Case-B recombination of He+ to He0 and of H+ to H0 have nearly equal coefficients at
    5e3..2e4 K (both ~2.6e-13 cm^3/s at 1e4 K; Osterbrock & Ferland 2006, Tables 2.1 and 2.4):
    the HeII fit lies within 10% of the hydrogen fit there."""
    T = np.array([5e3, 1e4, 2e4])
    t = cl.closure_terms(T)
    np.testing.assert_allclose(t["alpha_HeII_B"] / t["alpha_HII_B"], 1.0, rtol=0.1)
