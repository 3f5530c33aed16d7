"""The per-element comparison used by the GPU-against-oracle tests, checked on the CPU."""
import numpy as np

from parity import field_errors, fractions, rel_error


def test_faint_cell_error_is_seen():
    """A 1e-6 relative error in a cell eight decades below the brightest one passes a
    normwise 1e-10 bound but not the per-element one."""
    ref = np.array([1.0, 1e-8, 0.5])
    got = ref.copy()
    got[1] *= 1.0 + 1e-6
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-10
    assert rel_error(got, ref) > 1e-7


def test_floor_holds_cells_below_it_absolutely():
    """Below 1e-12 of the field's maximum a cell is held to an absolute 1e-12 max|ref|."""
    ref = np.array([1.0, 1e-20])
    got = np.array([1.0, 2e-20])
    assert rel_error(got, ref) < 1e-7


def test_fractions_of_each_element_sum_to_one():
    rng = np.random.default_rng(0)
    nH = rng.uniform(1e-4, 1e-2, 50)
    y = 0.0789
    n = np.stack([nH * rng.random(50), y * nH * 0.3 * rng.random(50), y * nH * 0.3 * rng.random(50)])
    f = fractions(n, nH, y)
    np.testing.assert_allclose(f["x_HI"] + f["x_HII"], 1.0, rtol=1e-14)
    np.testing.assert_allclose(f["x_HeI"] + f["x_HeII"] + f["x_HeIII"], 1.0, rtol=1e-14)


def test_ionised_cell_neutral_fraction_is_compared_on_its_own_scale():
    """n_HI = 1e-6 n_H off by 1e-4 relative: invisible under a normwise bound on n, seen on
    x_HI; the mask restricts the comparison (and its floor) to the given cells."""
    nH = np.array([1e-3, 1e-3])
    ref = {"E": np.ones(2), "e": np.ones(2), "n": np.array([[1e-3 * (1 - 1e-4), 1e-9]])}
    got = {"E": np.ones(2), "e": np.ones(2), "n": np.array([[1e-3 * (1 - 1e-4), 1e-9 * (1 + 1e-4)]])}
    err = field_errors(got, ref, nH)
    assert err["x_HI"] > 5e-5 and err["E"] == 0.0
    err = field_errors(got, ref, nH, mask=np.array([True, False]))
    assert err["x_HI"] == 0.0


def test_two_exact_oracle_solves_differ_within_the_newton_resolution():
    """The reading behind E's allowance: the same two steps solved two exact ways (D lagged with
    sparse LU of the whole Newton matrix; the exact Newton matrix with the Schur complement and
    BiCGStab), both to ||f|| < 1e-14, differ in faint cells by more than 1e-10 of the cell, but
    by less than 1e-14 u_E, the resolution the stopping test gives E; with that allowance the
    per-element comparison passes at 1e-10."""
    from conftest import oracle_problem
    from oracle import solve as sv
    from paper_0901_1110_gb300 import inputs
    from parity import TIGHT_NEWTON_TOL

    bc = ("dirichlet", "dirichlet", "zero_flux", "zero_flux", "periodic", "periodic")
    w = inputs.uniform_h(6, shape=(5, 6, 7), box=60 * inputs.KPC, dt=3e12, E0=1e-19, bc=bc)
    w.bc_value = (5e-16, 1e-18, 0.0, 0.0, 0.0, 0.0)
    w.theta = 1.0
    w.u_E = 1e-17
    out = []
    for lj, lin in (("lagged", "direct"), ("exact", "schur_cg")):
        p = oracle_problem(w, limiter_jacobian=lj)
        st = w.state()
        for _ in range(2):
            st, info = sv.implicit_step(p, st, w.dt, 1.0, 0.0, TIGHT_NEWTON_TOL, linear=lin)
            assert info["converged"]
        out.append(st)
    a, b = np.asarray(out[0]["E"]), np.asarray(out[1]["E"])
    assert rel_error(a, b) > 1e-10
    assert np.abs(a - b).max() <= TIGHT_NEWTON_TOL * w.u_E
    err = field_errors(out[0], out[1], w.nH, w.y_he, scales=(w.u_e, w.u_n, w.u_E))
    assert max(err.values()) <= 1e-10, err
