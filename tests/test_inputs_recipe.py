"""The synthetic workloads hold their stated recipe: the lognormal H + He medium (unit-variance
Gaussian field with P(k) ~ k^-2 and no k = 0 mode, n_H = nbar exp(sigma g - sigma^2 / 2)), the
helium ratio of Y = 0.24, the lognormal source rates, the uniform hydrogen benchmark, and
determinism in the seed."""
import numpy as np
import pytest

from paper_0901_1110_gb300 import inputs


def _radial_power(g):
    """Shell-averaged |FFT|^2 of g against |k| (cycles per cell)."""
    F = np.abs(np.fft.fftn(g)) ** 2
    kz, ky, kx = np.meshgrid(*(np.fft.fftfreq(n) for n in g.shape), indexing="ij")
    k = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    edges = np.linspace(0.02, 0.5, 25)
    idx = np.digitize(k.ravel(), edges)
    kc, pk = [], []
    for b in range(1, len(edges)):
        m = idx == b
        if m.any():
            kc.append(k.ravel()[m].mean())
            pk.append(F.ravel()[m].mean())
    return np.array(kc), np.array(pk)


def test_gaussian_field_is_unit_variance_with_a_k_minus_2_spectrum():
    g = inputs.gaussian_random_field((48, 48, 48), seed=3)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.0) < 1e-12
    assert abs(np.fft.fftn(g)[0, 0, 0]) < 1e-9                 # no k = 0 mode
    k, pk = _radial_power(g)
    slope = np.polyfit(np.log(k), np.log(pk), 1)[0]
    assert -2.2 < slope < -1.8, slope
    # another slope is honoured too
    k2, pk2 = _radial_power(inputs.gaussian_random_field((48, 48, 48), seed=3, slope=-1.0))
    assert -1.2 < np.polyfit(np.log(k2), np.log(pk2), 1)[0] < -0.8


def test_lognormal_medium_mean_dispersion_and_helium():
    w = inputs.lognormal_hhe((40, 44, 48), seed=5, nsrc=8)
    ln = np.log(w.nH / 1e-3)
    assert np.std(ln) == pytest.approx(1.0, rel=1e-9)           # sigma_ln (unit-variance g)
    assert np.mean(ln) == pytest.approx(-0.5, abs=1e-9)         # -sigma^2 / 2
    assert np.mean(w.nH) == pytest.approx(1e-3, rel=0.15)       # nbar, up to sample variance
    assert w.y_he == pytest.approx(0.24 / (4 * 0.76), rel=1e-12)
    nHI, nHeI, nHeII = w.n
    nHe = w.y_he * w.nH
    # x0 = 1e-4 of each element ionised, helium mostly singly
    assert np.allclose(w.nH - nHI, 1e-4 * w.nH, rtol=1e-9)
    assert np.all(nHeI + nHeII < nHe) and np.all(nHeI > 0.999 * nHe)
    assert np.all(w.E == 1e-20) and w.spectrum == ("blackbody", 1e5)


def test_source_rates_are_lognormal_with_the_stated_median():
    w = inputs.lognormal_hhe((8, 8, 8), seed=1, nsrc=4000)
    lr = np.log(w.src_rate / 1e49)
    assert abs(np.median(lr)) < 0.08 and abs(np.std(lr) - 1.0) < 0.05
    assert np.all((w.src_ijk >= 0) & (w.src_ijk < 8))


def test_uniform_benchmark_centre_source_and_state():
    w = inputs.config_uniform_32()
    assert (w.nx, w.ny, w.nz, w.ns) == (32, 32, 32, 1)
    assert w.dx == pytest.approx(inputs.MPC / 32)
    # 5e48 photons/s split over the 8 cells around the centre
    assert len(w.src_ijk) == 8 and w.src_rate.sum() == pytest.approx(5e48)
    assert {tuple(x) for x in w.src_ijk} == {(i, j, k) for i in (15, 16) for j in (15, 16)
                                             for k in (15, 16)}
    assert np.allclose(w.nH, 1e-3) and np.allclose(w.nH - w.n[0], 1e-7)
    assert (w.dt, w.nsteps, w.newton_tol, w.lin_tol) == (1e12, 5, 1e-8, 1e-10)


def test_workloads_are_deterministic_in_the_seed():
    a = inputs.config_lognormal(16, nsrc=4, seed=9)
    b = inputs.config_lognormal(16, nsrc=4, seed=9)
    assert np.array_equal(a.nH, b.nH) and np.array_equal(a.src_ijk, b.src_ijk)
    assert np.array_equal(a.src_rate, b.src_rate) and np.array_equal(a.e, b.e)
