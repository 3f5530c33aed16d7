"""Pins of the numpy V-cycle restatement (``mg_reference.py``) that the GPU multigrid is
compared with: the operator, the coarse operators and the restriction against brute-force
loops over cells written from their definitions, and the cycle's symmetry and positivity
(a fixed symmetric positive operator is what CG needs of a preconditioner, Sec. 3.2.2)."""
import numpy as np
import pytest

import mg_reference as mgr


def _random_operator(shape, periodic, seed):
    """Positive face entries (0 on zero-flux boundary faces) and a diagonal that dominates."""
    rng = np.random.default_rng(seed)
    W = [rng.uniform(0.1, 3.0, size=shape) for _ in range(3)]
    if not periodic:
        W[0][:, :, 0] = 0.0
        W[1][:, 0, :] = 0.0
        W[2][0, :, :] = 0.0
    loc = rng.uniform(0.5, 2.0, size=shape)
    return loc + mgr.face_sum(W), W


def _neighbours(shape, periodic, k, j, i):
    """(lower-face entry index, lower neighbour, upper-face entry index, upper neighbour) per
    axis; None where a zero-flux boundary has no neighbour."""
    nz, ny, nx = shape
    out = []
    for ax, (q, n) in enumerate(((i, nx), (j, ny), (k, nz))):
        def cell(v):
            if ax == 0:
                return (k, j, v)
            if ax == 1:
                return (k, v, i)
            return (v, j, i)
        lo = cell(q - 1) if q > 0 else (cell(n - 1) if periodic else None)
        hi = cell(q + 1) if q < n - 1 else (cell(0) if periodic else None)
        out.append((ax, lo, hi, cell(q + 1) if q < n - 1 else cell(0)))
    return out


def _apply_loops(d, W, x, periodic, Wp=None):
    """Row c: d x_c - (its lower face's W) x_lo - (its upper face's Wp) x_hi, per axis."""
    Wp = W if Wp is None else Wp
    shape = d.shape
    y = np.zeros_like(x)
    for k in range(shape[0]):
        for j in range(shape[1]):
            for i in range(shape[2]):
                v = d[k, j, i] * x[k, j, i]
                for ax, lo, hi, hi_face in _neighbours(shape, periodic, k, j, i):
                    if lo is not None:
                        v -= W[ax][k, j, i] * x[lo]
                    if hi is not None:
                        v -= Wp[ax][hi_face] * x[hi]
                y[k, j, i] = v
    return y


def _coarsen_loops_nonsym(d, W, Wp, periodic):
    """Coarse operator of a non-symmetric operator from its definition, loop by loop."""
    shape = d.shape
    cs = tuple((n + 1) // 2 for n in shape)
    dc = np.zeros(cs)
    Wc = [np.zeros(cs) for _ in range(3)]
    Wpc = [np.zeros(cs) for _ in range(3)]
    for K, J, I in np.ndindex(*cs):
        loc, cnt = 0.0, 0
        fs, fp, fc = [0.0] * 3, [0.0] * 3, [0] * 3
        for dk, dj, di in np.ndindex(2, 2, 2):
            k, j, i = 2 * K + dk, 2 * J + dj, 2 * I + di
            if k >= shape[0] or j >= shape[1] or i >= shape[2]:
                continue
            row = 0.0
            for ax, lo, hi, hi_face in _neighbours(shape, periodic, k, j, i):
                row += W[ax][k, j, i]
                if hi is not None:
                    row += Wp[ax][hi_face]
            loc += d[k, j, i] - row
            cnt += 1
            for ax, first in enumerate((di == 0, dj == 0, dk == 0)):
                if first:
                    fs[ax] += W[ax][k, j, i]
                    fp[ax] += Wp[ax][k, j, i]
                    fc[ax] += 1
        dc[K, J, I] = loc / cnt
        for ax in range(3):
            Wc[ax][K, J, I] = 0.25 * fs[ax] / fc[ax]
            Wpc[ax][K, J, I] = 0.25 * fp[ax] / fc[ax]
    for K, J, I in np.ndindex(*cs):
        for ax, lo, hi, hi_face in _neighbours(cs, periodic, K, J, I):
            dc[K, J, I] += Wc[ax][K, J, I]
            if hi is not None:
                dc[K, J, I] += Wpc[ax][hi_face]
    return dc, Wc, Wpc


def _coarsen_loops(d, W, periodic):
    shape = d.shape
    cs = tuple((n + 1) // 2 for n in shape)
    dc = np.zeros(cs)
    Wc = [np.zeros(cs) for _ in range(3)]
    for K in range(cs[0]):
        for J in range(cs[1]):
            for I in range(cs[2]):
                loc, cnt = 0.0, 0
                fs = [0.0, 0.0, 0.0]
                fc = [0, 0, 0]
                for dk in range(2):
                    for dj in range(2):
                        for di in range(2):
                            k, j, i = 2 * K + dk, 2 * J + dj, 2 * I + di
                            if k >= shape[0] or j >= shape[1] or i >= shape[2]:
                                continue
                            six = 0.0
                            for ax, lo, hi, hi_face in _neighbours(shape, periodic, k, j, i):
                                six += W[ax][k, j, i]
                                if hi is not None:
                                    six += W[ax][hi_face]
                            loc += d[k, j, i] - six
                            cnt += 1
                            for ax, first in enumerate((di == 0, dj == 0, dk == 0)):
                                if first:
                                    fs[ax] += W[ax][k, j, i]
                                    fc[ax] += 1
                dc[K, J, I] = loc / cnt
                for ax in range(3):
                    Wc[ax][K, J, I] = 0.25 * fs[ax] / fc[ax]
    # diagonal = local diagonal + the six coarse face entries
    for K in range(cs[0]):
        for J in range(cs[1]):
            for I in range(cs[2]):
                for ax, lo, hi, hi_face in _neighbours(cs, periodic, K, J, I):
                    dc[K, J, I] += Wc[ax][K, J, I]
                    if hi is not None:
                        dc[K, J, I] += Wc[ax][hi_face]
    return dc, Wc


@pytest.mark.parametrize("periodic", [False, True])
def test_apply_matches_loops(periodic):
    d, W = _random_operator((3, 4, 5), periodic, 1)
    x = np.random.default_rng(2).standard_normal(d.shape)
    np.testing.assert_allclose(mgr.apply(d, W, x), _apply_loops(d, W, x, periodic),
                               rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("shape", [(4, 6, 8), (5, 6, 7), (1, 3, 2)])
def test_coarsen_matches_loops(periodic, shape):
    d, W = _random_operator(shape, periodic, 3)
    cs = mgr.levels(shape, 2)[1]
    dc, Wc = mgr.coarsen(d, W, cs)
    dl, Wl = _coarsen_loops(d, W, periodic)
    np.testing.assert_allclose(dc, dl, rtol=1e-13)
    for ax in range(3):
        np.testing.assert_allclose(Wc[ax], Wl[ax], rtol=1e-13, atol=1e-15)


def test_restriction_is_the_children_sum_over_8():
    rng = np.random.default_rng(4)
    F = rng.standard_normal((5, 6, 7))
    cs = mgr.levels(F.shape, 2)[1]
    R = mgr.restrict(F, cs)
    for K, J, I in np.ndindex(*cs):
        kids = F[2 * K:2 * K + 2, 2 * J:2 * J + 2, 2 * I:2 * I + 2]
        assert abs(R[K, J, I] - kids.sum() / 8) <= 1e-14


def test_levels_round_up_and_stop_at_one_cell():
    assert mgr.levels((18, 20, 24), 4) == [(18, 20, 24), (9, 10, 12), (5, 5, 6), (3, 3, 3)]
    assert mgr.levels((3, 1, 2), 6) == [(3, 1, 2), (2, 1, 1), (1, 1, 1)]


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 7, 9), (5, 8, 2)])
def test_vcycle_is_symmetric_positive_and_contracts(periodic, shape):
    """With equal pre- and post-sweeps the cycle is a symmetric positive operator M, also on
    odd extents, and x <- x + M (b - A x) converges."""
    d, W = _random_operator(shape, periodic, 5)
    ops = mgr.hierarchy(d, W, 3)
    rng = np.random.default_rng(6)
    a, b = rng.standard_normal(d.shape), rng.standard_normal(d.shape)

    def M(v):
        return mgr.vcycle(ops, v, 0.9, 2, 2, 16)

    Ma, Mb = M(a), M(b)
    assert abs(np.vdot(b, Ma) - np.vdot(a, Mb)) <= 1e-12 * np.sqrt(np.vdot(a, Ma) * np.vdot(b, Mb))
    assert np.vdot(a, Ma) > 0 and np.vdot(b, Mb) > 0
    x = np.zeros_like(b)
    r0 = np.linalg.norm(b)
    for _ in range(10):
        x = x + M(b - mgr.apply(d, W, x))
    assert np.linalg.norm(b - mgr.apply(d, W, x)) < 1e-3 * r0


def _random_nonsym(shape, periodic, seed):
    """Non-symmetric couplings: Wp = W times a factor in [0.5, 1.5], diagonally dominant rows."""
    d, W = _random_operator(shape, periodic, seed)
    rng = np.random.default_rng(seed + 100)
    Wp = [w * rng.uniform(0.5, 1.5, size=shape) for w in W]
    return d + mgr.face_sum(W, Wp) - mgr.face_sum(W), W, Wp


@pytest.mark.parametrize("periodic", [False, True])
def test_nonsymmetric_apply_matches_loops(periodic):
    d, W, Wp = _random_nonsym((3, 4, 5), periodic, 7)
    x = np.random.default_rng(8).standard_normal(d.shape)
    np.testing.assert_allclose(mgr.apply(d, W, x, Wp), _apply_loops(d, W, x, periodic, Wp),
                               rtol=1e-13, atol=1e-13)
    # the symmetric form is the special case Wp = W
    np.testing.assert_array_equal(mgr.apply(d, W, x, W), mgr.apply(d, W, x))


@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("shape", [(4, 6, 8), (5, 6, 7), (1, 3, 2)])
def test_nonsymmetric_coarsen_matches_loops(periodic, shape):
    d, W, Wp = _random_nonsym(shape, periodic, 9)
    cs = mgr.levels(shape, 2)[1]
    dc, Wc, Wpc = mgr.coarsen(d, W, cs, Wp)
    dl, Wl, Wpl = _coarsen_loops_nonsym(d, W, Wp, periodic)
    np.testing.assert_allclose(dc, dl, rtol=1e-13)
    for ax in range(3):
        np.testing.assert_allclose(Wc[ax], Wl[ax], rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(Wpc[ax], Wpl[ax], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 7, 9)])
def test_nonsymmetric_vcycle_contracts(shape):
    """The cycle of a non-symmetric diagonally dominant operator reduces the residual of
    x <- x + M (b - A x) as the symmetric one does."""
    d, W, Wp = _random_nonsym(shape, False, 11)
    ops = mgr.hierarchy(d, W, 3, Wp)
    assert all(len(o) == 3 for o in ops)
    b = np.random.default_rng(12).standard_normal(d.shape)
    x = np.zeros_like(b)
    for _ in range(10):
        x = x + mgr.vcycle(ops, b - mgr.apply(d, W, x, Wp), 0.9, 2, 2, 16)
    assert np.linalg.norm(b - mgr.apply(d, W, x, Wp)) < 1e-3 * np.linalg.norm(b)
