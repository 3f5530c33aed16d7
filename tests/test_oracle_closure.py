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
