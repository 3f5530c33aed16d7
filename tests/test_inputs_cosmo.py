"""Host logic of the cosmological configuration: the flat Lambda-CDM expansion history and the
clustered source placement of the synthetic workload generator."""
import numpy as np
import pytest

from paper_0901_1110_gb300 import inputs


def test_flat_lcdm_history():
    """a(t) inverts t(a); da/dt = a H(a) (central differences); in the matter era
    a ~ t^(2/3); z = 10 -> 6 spans the textbook ~0.47 Gyr for Om = 0.3, H0 = 70."""
    a = np.array([1 / 11, 1 / 7, 0.5, 1.0])
    t = inputs.flat_lcdm_t(a)
    np.testing.assert_allclose(inputs.flat_lcdm_a(t), a, rtol=1e-13)
    h = 1e-6 * t
    fd = (inputs.flat_lcdm_a(t + h) - inputs.flat_lcdm_a(t - h)) / (2 * h)
    np.testing.assert_allclose(fd, inputs.flat_lcdm_adot(a), rtol=1e-8)
    r = inputs.flat_lcdm_a(2e15) / inputs.flat_lcdm_a(1e15)
    assert r == pytest.approx(2 ** (2 / 3), rel=1e-3)             # deep matter era
    gyr = 3.15576e16
    span = (inputs.flat_lcdm_t(1 / 7) - inputs.flat_lcdm_t(1 / 11)) / gyr
    assert 0.40 < span < 0.55
    assert inputs.flat_lcdm_t(1.0) / gyr == pytest.approx(13.47, rel=0.01)   # age today


def test_cosmological_configuration_small():
    w = inputs.config_cosmo(n=16, nsrc=12, nsteps=10)
    assert len(w.schedule) == 10 and w.theta == 1.0
    dts = [s[0] for s in w.schedule]
    assert np.allclose(dts, dts[0])
    a = np.array([s[1] for s in w.schedule])
    assert 1 / 11 < a[0] < a[-1] < 1 / 7 and np.all(np.diff(a) > 0)
    # sigma_ln = 1.5 and sources drawn ~ n_H^2 sit in dense cells
    assert np.std(np.log(w.nH)) == pytest.approx(1.5, rel=0.05)
    nsrc = w.nH[w.src_ijk[:, 2], w.src_ijk[:, 1], w.src_ijk[:, 0]]
    assert np.median(nsrc) > 3 * np.median(w.nH)
    assert len({tuple(x) for x in w.src_ijk}) == 12
