"""Pins of the oracle's residual, Jacobian, Schur reduction and Newton solve.

Each test checks the oracle against something other than itself: a closed-form solution of
a special case, a library diagonalisation, finite differences, or an exact discrete
conservation identity."""
import numpy as np
import pytest
from scipy import fft

from conftest import oracle_problem
from oracle import closure as cl, model as md, solve as sv
from paper_0901_1110_gb300 import inputs

KPC = inputs.KPC


def _random_state(p, rng, T_range=(50.0, 1e6), E_scale=1e-17):
    """A generic interior state of p's cells with temperatures spread over T_range."""
    ns = p.ns
    U = np.empty((p.nv, p.N))
    nHe = p.y_he * p.nH
    U[1] = p.nH * rng.uniform(0.05, 0.95, p.N)
    if ns == 3:
        f1 = rng.uniform(0.05, 0.9, p.N)
        f2 = rng.uniform(0.05, 0.95 - f1)
        U[2] = nHe * f1
        U[3] = nHe * f2
    U[1 + ns] = E_scale * rng.uniform(0.3, 3.0, p.N)
    nHI, nHeI, nHeII = p.species_full(U[1:1 + ns])
    _, _, ne = cl.derived_species(p.nH, nHe, nHI, nHeI, nHeII)
    T = np.exp(rng.uniform(np.log(T_range[0]), np.log(T_range[1]), p.N))
    e_total = T * cl.K_BOLTZ * (p.nH + nHe + ne) / ((cl.GAMMA - 1) * cl.mass_density(p.nH, nHe))
    eh = e_total * rng.uniform(0.6, 1.4, p.N)
    U[0] = e_total - eh
    return U, eh


def _fd_jacobian(p, U, g, eh, dt, a, adot, T_fixed, W=None, kap_faces=None):
    u = p.scales()
    Jfd = np.zeros((p.nv * p.N, p.nv * p.N))
    for v in range(p.nv):
        for c in range(p.N):
            h = 1e-6 * max(abs(U[v, c]), 1e-3 * u[v])
            Up = U.copy(); Up[v, c] += h
            Um = U.copy(); Um[v, c] -= h
            fp = md.residual(p, Up, g, eh, dt, a, adot, T_fixed, W=W, kap_faces=kap_faces) / u[:, None]
            fm = md.residual(p, Um, g, eh, dt, a, adot, T_fixed, W=W, kap_faces=kap_faces) / u[:, None]
            Jfd[:, v * p.N + c] = ((fp - fm) / (2 * h) * u[v]).ravel()
    return Jfd


@pytest.mark.parametrize("ns,isothermal,a,adot", [(1, False, 1.0, 0.0), (3, False, 1.0, 0.0),
                                                   (3, False, 0.2, 3e-17), (3, True, 0.5, 1e-17),
                                                   (1, True, 1.0, 0.0)])
def test_jacobian_matches_central_differences(ns, isothermal, a, adot):
    """Eqs. jacobian_matrix / jacobian_submatrices: the analytic Newton matrix equals central
    differences of f (eq. nonlinear_residual) with the face coefficients frozen (lagged D),
    over states from 50 K to 1e6 K, with cosmological a(t) terms, both species sets."""
    rng = np.random.default_rng(10 * ns + int(isothermal))
    if ns == 1:
        w = inputs.uniform_h(3, shape=(2, 3, 3), box=60 * KPC, dt=3e13)
    else:
        w = inputs.lognormal_hhe((2, 3, 3), box=60 * KPC, nsrc=2, dt=3e13)
    p = oracle_problem(w, rates=cl.SmoothRates(), isothermal=isothermal, theta=0.7)
    U, eh = _random_state(p, rng)
    Un = md.state_to_U(p, w.state())
    T_fixed = rng.uniform(100.0, 3e4, p.N) if isothermal else None
    g = md.build_g(p, Un, w.e.ravel(), w.dt, a, adot, T_fixed)
    lt = md.local_terms(p, U[0], U[1:1 + ns], U[1 + ns], eh, p.nH, p.src, a, adot, T_fixed)
    W = md.face_weights(p, U[1 + ns], lt["kappa"], a)
    J = md.full_jacobian(p, U, eh, w.dt, a, adot, T_fixed).toarray()
    Jfd = _fd_jacobian(p, U, g, eh, w.dt, a, adot, T_fixed, W)
    scale = np.abs(Jfd).max(axis=1, keepdims=True)
    assert np.max(np.abs(J - Jfd) / scale) < 1e-6


@pytest.mark.parametrize("ns", [1, 3])
def test_jacobian_with_dD_dE_matches_central_differences(ns):
    """Sec. 3.2.1: the Newton matrix that keeps the limiter's E dependence and lags only its
    opacity equals central differences of f with the face opacities frozen, including faces
    in the free-streaming regime (steep E contrasts, thin cells)."""
    rng = np.random.default_rng(40 + ns)
    if ns == 1:
        w = inputs.uniform_h(3, shape=(2, 3, 4), box=60 * KPC, dt=3e13, bc=("periodic",) * 6)
    else:
        w = inputs.lognormal_hhe((2, 3, 4), box=60 * KPC, nsrc=2, dt=3e13)
    p = oracle_problem(w, rates=cl.SmoothRates(), theta=0.8, limiter_jacobian="E")
    U, eh = _random_state(p, rng)
    U[1 + ns] = 1e-17 * np.exp(rng.uniform(-6.0, 6.0, p.N))     # strong gradients
    U[1] = p.nH * rng.uniform(1e-6, 1e-4, p.N)                   # ionised: optically thin
    if ns == 3:
        U[2] = p.y_he * p.nH * rng.uniform(1e-6, 1e-4, p.N)
    Un = md.state_to_U(p, w.state())
    g = md.build_g(p, Un, w.e.ravel(), w.dt, 1.0, 0.0)
    lt = md.local_terms(p, U[0], U[1:1 + ns], U[1 + ns], eh, p.nH, p.src, 1.0, 0.0)
    J = md.full_jacobian(p, U, eh, w.dt, 1.0, 0.0).toarray()
    Jfd = _fd_jacobian(p, U, g, eh, w.dt, 1.0, 0.0, None, kap_faces=lt["kappa"])
    scale = np.abs(Jfd).max(axis=1, keepdims=True)
    # the limiter is strongly nonlinear across these contrasts: central differences with a
    # 1e-6 step carry ~1e-6..1e-5 truncation error here; a wrong term shows up at O(1)
    assert np.max(np.abs(J - Jfd) / scale) < 3e-5
    # and it is not symmetric (the E block carries the limiter's advective part)
    nm = ns + 1
    JE = J[nm * p.N:, nm * p.N:]
    off = JE - np.diag(np.diag(JE))
    assert np.abs(off - off.T).max() > 1e-2 * np.abs(off).max()


@pytest.mark.parametrize("ns,limiter", [(1, True), (3, True), (3, False)])
def test_exact_jacobian_matches_central_differences(ns, limiter):
    """The exact Newton matrix (dD/dE and the opacity's species dependence kept) equals central
    differences of f with nothing frozen, including the E-row entries in the species columns
    of the neighbours; ionised thin cells with steep E contrasts and neutral thick ones."""
    rng = np.random.default_rng(70 + ns)
    if ns == 1:
        w = inputs.uniform_h(3, shape=(2, 3, 4), box=60 * KPC, dt=3e13, bc=("periodic",) * 6)
    else:
        w = inputs.lognormal_hhe((2, 3, 4), box=60 * KPC, nsrc=2, dt=3e13)
    p = oracle_problem(w, rates=cl.SmoothRates(), theta=0.8, limiter_jacobian="exact",
                       limiter=limiter)
    U, eh = _random_state(p, rng)
    U[1 + ns] = 1e-17 * np.exp(rng.uniform(-6.0, 6.0, p.N))
    U[1] = p.nH * np.where(rng.random(p.N) < 0.5, rng.uniform(1e-6, 1e-4, p.N),
                           rng.uniform(0.3, 0.99, p.N))
    if ns == 3:
        U[2] = p.y_he * p.nH * rng.uniform(1e-6, 0.5, p.N)
        U[3] = p.y_he * p.nH * rng.uniform(1e-6, 0.4, p.N)
    Un = md.state_to_U(p, w.state())
    g = md.build_g(p, Un, w.e.ravel(), w.dt, 1.0, 0.0)
    J = md.full_jacobian(p, U, eh, w.dt, 1.0, 0.0).toarray()
    Jfd = _fd_jacobian(p, U, g, eh, w.dt, 1.0, 0.0, None)
    scale = np.abs(Jfd).max(axis=1, keepdims=True)
    assert np.max(np.abs(J - Jfd) / scale) < 3e-5
    # the species columns of the E rows reach the neighbours
    nm = ns + 1
    JEn = J[nm * p.N:, p.N:2 * p.N]
    assert np.count_nonzero(JEn - np.diag(np.diag(JEn))) > 0


def test_limiter_limits():
    """Eq. limiter: D -> c/(3 kappa) as R -> 0 (diffusion) and D R -> c as R -> inf
    (free streaming, flux |F| = c E)."""
    p = oracle_problem(inputs.uniform_h(2))
    kap = np.array([2e-21])
    Ea = np.array([1.0])
    for Eb, want in ((1.0 + 1e-9, cl.C_LIGHT / (3 * kap[0]) / p.dx ** 2),):
        got = md.face_coefficient(p, Ea, np.array([Eb]), kap, kap, 1.0)[0]
        assert abs(got / want - 1) < 1e-8
    Eb = np.array([1e-12])
    R = np.abs(Eb - Ea) / (p.dx * 0.5 * (Ea + Eb))
    D = md.face_coefficient(p, Ea, Eb, kap * 1e-12, kap * 1e-12, 1.0) * p.dx ** 2
    assert abs(D[0] * R[0] / cl.C_LIGHT - 1) < 1e-6
    # transparent medium with a flat field: D = c / R_min = c a L
    D0 = md.face_coefficient(p, Ea, Ea, 0 * kap, 0 * kap, 0.5) * (0.5 * p.dx) ** 2
    assert abs(D0[0] / (cl.C_LIGHT * 0.5 * 2 * p.dx) - 1) < 1e-14
    # symmetric in the two cells
    D1 = md.face_coefficient(p, np.array([2.0]), np.array([3.0]), kap, 2 * kap, 1.0)
    D2 = md.face_coefficient(p, np.array([3.0]), np.array([2.0]), 2 * kap, kap, 1.0)
    assert D1[0] == D2[0]


def _pure_diffusion_problem(n_shape, bc, theta):
    nz, ny, nx = n_shape
    dx = 4e21               # with sigma = 6.3e-21: dt W ~ 0.1 and every mode decays monotonically
    w = inputs.uniform_h(nx, shape=n_shape, box=nx * dx, x0=0.0, dt=1e9,
                         bc=(bc,) * 6)
    w.theta = theta
    grey = dict(sk=np.array([6.3e-21, 0, 0]), pgam=np.zeros(3), ph=np.zeros(3))
    p = oracle_problem(w, grey=grey, limiter=False, src=np.zeros(w.N), u_E=1e-17)
    rng = np.random.default_rng(3)
    st = w.state()
    st["E"] = 1e-17 * rng.uniform(0.2, 2.0, w.N)
    return w, p, st


@pytest.mark.parametrize("bc", ["zero_flux", "periodic"])
@pytest.mark.parametrize("theta", [1.0, 0.51])
def test_diffusion_step_equals_discrete_exact_solution(bc, theta):
    """Eqs. radiation_simplified + mDE with constant kappa and no reactions: one theta step
    is diagonalised exactly by the DCT-II (zero-flux faces) or the DFT (periodic)."""
    shape = (5, 6, 7)
    w, p, st = _pure_diffusion_problem(shape, bc, theta)
    new, stats = sv.implicit_step(p, st, w.dt, 1.0, 0.0, 1e-13, linear="direct")
    assert stats["converged"]
    kap = 6.3e-21 * p.nH[0]
    Wc = cl.C_LIGHT / (3 * kap) / p.dx ** 2
    E0 = st["E"].reshape(shape)
    lam = 0.0
    for ax, n in enumerate(shape):
        k = np.arange(n)
        ev = 2 - 2 * np.cos(np.pi * k / n) if bc == "zero_flux" else 2 - 2 * np.cos(2 * np.pi * k / n)
        sh = [1, 1, 1]; sh[ax] = n
        lam = lam + ev.reshape(sh)
    A = Wc * lam + cl.C_LIGHT * kap
    amp = (1 - w.dt * (1 - theta) * A) / (1 + w.dt * theta * A)
    if bc == "zero_flux":
        E1 = fft.idctn(fft.dctn(E0, type=2, norm="ortho") * amp, type=2, norm="ortho")
    else:
        E1 = np.real(np.fft.ifftn(np.fft.fftn(E0) * amp))
    np.testing.assert_allclose(new["E"].reshape(shape), E1, rtol=1e-11, atol=1e-11 * E1.max())
    np.testing.assert_allclose(new["n"], st["n"], rtol=1e-14)


def _gaussian_pulse_error(n, nsteps):
    """Max error, relative to the peak, of theta = 1 steps of a Gaussian pulse in a periodic
    box (constant kappa, no reactions, limiter off) against the analytic solution."""
    L, nH = 4.8e22, 1e-3
    sig0 = L / 8                       # periodic images sit 8 sigma0 away: exp(-16) at the end
    kap = 6.3e-21 * nH
    D = cl.C_LIGHT / (3 * kap)
    T = sig0 ** 2 / (2 * D)            # sigma^2 doubles
    dt = T / nsteps
    w = inputs.uniform_h(n, shape=(n, n, n), box=L, x0=0.0, dt=dt, bc=("periodic",) * 6, nH=nH)
    w.theta = 1.0
    grey = dict(sk=np.array([6.3e-21, 0, 0]), pgam=np.zeros(3), ph=np.zeros(3))
    p = oracle_problem(w, grey=grey, limiter=False, src=np.zeros(w.N), u_E=1e-17)
    st = w.state()
    x = (np.arange(n) + 0.5) * (L / n) - L / 2
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    r2 = X ** 2 + Y ** 2 + Z ** 2
    bg, E0 = 1e-20, 1e-17
    st["E"] = (bg + E0 * np.exp(-r2 / (2 * sig0 ** 2))).ravel()
    for _ in range(nsteps):
        st, stats = sv.implicit_step(p, st, dt, 1.0, 0.0, 1e-13, linear="schur_cg")
        assert stats["converged"]
    s2 = sig0 ** 2 + 2 * D * T
    exact = np.exp(-cl.C_LIGHT * kap * T) * (bg + E0 * (sig0 ** 2 / s2) ** 1.5
                                             * np.exp(-r2 / (2 * s2)))
    return np.abs(st["E"].reshape(n, n, n) - exact).max() / exact.max()


def test_gaussian_pulse_converges_to_the_heat_kernel():
    """Eqs. radiation_simplified + mDE in the diffusion limit, D = c / (3 kappa), against the
    analytic solution of dE/dt = D lap E - c kappa E for a Gaussian pulse:
    E = exp(-c kappa t) (s0^2 / s^2)^(3/2) exp(-r^2 / (2 s^2)), s^2 = s0^2 + 2 D t.
    With theta = 1 the error is O(dx^2 + dt): halving dx and quartering dt cuts it by about 4."""
    coarse = _gaussian_pulse_error(24, 8)
    fine = _gaussian_pulse_error(48, 32)
    assert fine < 0.025
    assert 3.3 < coarse / fine < 4.7, (coarse, fine)


@pytest.mark.parametrize("limiter", [False, True])
def test_comoving_grid_is_the_proper_grid(limiter):
    """Reading of the comoving factors: diffusion (1/a^2) div(D grad E) with R = |grad E| /
    (a E), opacities from proper densities n / a^3.  A comoving grid of spacing dx at scale
    factor a (adot = 0) is then the proper grid of spacing a dx holding the proper densities,
    so one step of the radiation equation (no sources, no photo-absorption by species) gives
    the same E on both."""
    shape = (5, 6, 7)
    nz, ny, nx = shape
    a = 0.5
    E0 = 1e-17 * np.exp(np.random.default_rng(3).uniform(-3.0, 3.0, nx * ny * nz))
    out = []
    for scale, dx, nH in ((a, 4e21, 1e-3), (1.0, a * 4e21, 1e-3 / a ** 3)):
        w = inputs.uniform_h(nx, shape=shape, box=nx * dx, x0=0.0, dt=1e9, nH=nH,
                             bc=("zero_flux",) * 6)
        w.theta = 1.0
        grey = dict(sk=np.array([6.3e-21, 0, 0]), pgam=np.zeros(3), ph=np.zeros(3))
        p = oracle_problem(w, grey=grey, limiter=limiter, src=np.zeros(w.N), u_E=1e-17)
        st = w.state()
        st["E"] = E0.copy()
        new, stats = sv.implicit_step(p, st, w.dt, scale, 0.0, 1e-13, linear="direct")
        assert stats["converged"]
        out.append(np.asarray(new["E"]))
    np.testing.assert_allclose(out[0], out[1], rtol=1e-10, atol=0)
    assert np.abs(out[0] / E0 - 1).max() > 1e-2          # the step did move E


@pytest.mark.parametrize("theta", [1.0, 0.51])
def test_expansion_terms_closed_form(theta):
    """The cosmological terms -m (adot/a) E (eq. mLE) and -2 (adot/a) e_c (eq. mLe) in a
    uniform neutral medium with photoheating but no absorption or ionisation: the theta
    step has the closed forms E' = E (1 - (1-theta) dt H) / (1 + theta dt H) and
    e_c (1 + 2 theta dt H) = dt (theta G(E') + (1-theta) G(E))."""
    a, H = 0.25, 2e-17
    adot = a * H
    w = inputs.uniform_h(3, x0=0.0, dt=3e15, bc=("periodic",) * 6, E0=1e-16)
    w.theta = theta
    grey = dict(sk=np.zeros(3), pgam=np.zeros(3), ph=np.array([2e-25, 0, 0]))
    p = oracle_problem(w, grey=grey, src=np.zeros(w.N), u_E=1e-16)
    st = w.state()
    new, stats = sv.implicit_step(p, st, w.dt, a, adot, 1e-13)
    assert stats["converged"]
    E0 = st["E"][0]
    E1 = E0 * (1 - (1 - theta) * w.dt * H) / (1 + theta * w.dt * H)
    np.testing.assert_allclose(new["E"], E1, rtol=1e-13)
    rho = cl.M_H * p.nH[0]
    G = lambda E: cl.C_LIGHT * E / a ** 3 * grey["ph"][0] * p.nH[0] / rho
    ec = w.dt * (theta * G(E1) + (1 - theta) * G(E0)) / (1 + 2 * theta * w.dt * H)
    np.testing.assert_allclose(new["e"] - st["e"], ec, rtol=1e-12)


def test_photoionisation_equilibrium_closed_form():
    """Hydrogen at fixed T = 1e4 K (as in Sec. 4.5) under a constant photoionisation rate:
    long backward-Euler steps reach (alpha + beta) n_H x^2 + (Gamma - beta n_H) x - Gamma = 0,
    i.e. x^2 / (1 - x) = Gamma / (n_H alpha_B) when collisions are negligible."""
    nH = 1e-3
    w = inputs.uniform_h(2, T0=1e4, x0=0.5, nH=nH, bc=("periodic",) * 6, dt=1e18)
    w.theta = 1.0
    grey = cl.grey_constants("mono", 13.6 * cl.EV, 1)
    Gamma = 2e-13
    E0 = Gamma / (cl.C_LIGHT * grey["pgam"][0])
    k, _ = cl.RateTable()(np.array([1e4]))
    al, be = k[0, 0], k[0, 1]
    A, B, C = (al + be) * nH, Gamma - be * nH, -Gamma
    x = (-B + np.sqrt(B * B - 4 * A * C)) / (2 * A)
    src = np.full(w.N, cl.C_LIGHT * grey["sk"][0] * nH * (1 - x) * E0)
    p = oracle_problem(w, grey=grey, src=src, isothermal=True, u_E=E0, u_n=nH)
    st = w.state()
    st["E"][:] = E0
    for _ in range(8):
        st, stats = sv.implicit_step(p, st, w.dt, 1.0, 0.0, 1e-10)
        assert stats["converged"]
    xHII = 1 - st["n"][0] / nH
    np.testing.assert_allclose(xHII, x, rtol=1e-11)
    np.testing.assert_allclose(st["n"][0], nH * (1 - x), rtol=1e-8)     # the small n_HI too
    np.testing.assert_allclose(st["E"], E0, rtol=1e-8)
    assert abs(x * x / (1 - x) / (Gamma / (nH * al)) - 1) < 1e-3   # collisions negligible


@pytest.mark.parametrize("theta", [1.0, 0.6])
def test_photon_number_conservation_periodic_box(theta):
    """In a periodic box with monochromatic 13.6 eV photons every absorbed photon ionises
    one atom and diffusion only moves photons, so the theta scheme conserves
    sum(E / h nu + n_HII) up to the sources and the theta-weighted two-body terms:
    Delta = dt sum(src / h nu + theta R^{n+1} + (1 - theta) R^n), R = n_e (beta n_HI - alpha n_HII)."""
    w = inputs.uniform_h(6, shape=(4, 5, 6), box=120 * KPC, dt=5e9, x0=0.2, T0=8e3,
                         bc=("periodic",) * 6, ndot=3e49)
    w.theta = theta
    rng = np.random.default_rng(5)
    w.nH = w.nH * rng.uniform(0.5, 1.5, w.nH.shape)
    w.n = (0.8 * w.nH)[None]
    p = oracle_problem(w, u_E=1e-17)
    hnu = 13.6 * cl.EV
    st = w.state()
    st["E"] = 1e-17 * rng.uniform(0.5, 2.0, w.N)

    def R(state):
        nHI = state["n"][0]
        nHII = p.nH - nHI
        T = md.fixed_temperature(p, state)
        k, _ = p.rates(T)
        return nHII * (k[:, 1] * nHI - k[:, 0] * nHII)

    new, stats = sv.implicit_step(p, st, w.dt, 1.0, 0.0, 1e-12, linear="direct")
    assert stats["converged"]
    count = lambda s: np.sum(s["E"] / hnu + (p.nH - s["n"][0]))
    lhs = count(new) - count(st)
    rhs = w.dt * np.sum(p.src / hnu + theta * R(new) + (1 - theta) * R(st))
    assert abs(lhs - rhs) <= 1e-10 * count(st)
    photons = lambda s: np.sum(s["E"] / hnu)
    assert abs(photons(new) - photons(st)) > 1e-3 * photons(st)   # photons were absorbed


@pytest.mark.parametrize("ljac", ["lagged", "E", "exact"])
@pytest.mark.parametrize("ns,bc", [(1, "zero_flux"), (3, "zero_flux"), (3, "periodic")])
def test_schur_reduction_equals_unreduced_solve(ns, bc, ljac):
    """Sec. 3.2.1 steps (i)-(iii) (eqs. newton_system2, schur_components, step_ia) give the
    same Newton correction as a direct solve of the whole unreduced system."""
    rng = np.random.default_rng(ns)
    if ns == 1:
        w = inputs.uniform_h(4, shape=(3, 4, 5), box=80 * KPC, dt=3e13, bc=(bc,) * 6)
    else:
        w = inputs.lognormal_hhe((3, 4, 5), box=80 * KPC, nsrc=2, dt=3e13, bc=(bc,) * 6)
    w.theta = 0.8
    p = oracle_problem(w, limiter_jacobian=ljac)
    U, eh = _random_state(p, rng, T_range=(100, 1e5))
    Un = md.state_to_U(p, w.state())
    g = md.build_g(p, Un, w.e.ravel(), w.dt, 1.0, 0.0)
    f = md.residual(p, U, g, eh, w.dt, 1.0, 0.0)
    s_direct, _ = sv.newton_direction(p, U, f, eh, w.dt, 1.0, 0.0, linear="direct")
    s_schur, _ = sv.newton_direction(p, U, f, eh, w.dt, 1.0, 0.0, linear="schur_direct")
    s_cg, _ = sv.newton_direction(p, U, f, eh, w.dt, 1.0, 0.0, linear="schur_cg")
    u = p.scales()[:, None]
    ref = np.abs(s_direct / u).max()
    # the exact matrix couples E to the neighbours' species and is worse conditioned on these
    # random states (steps of 1e13 in scaled units): roundoff reaches a few 1e-10 there
    tol = 1e-11 if ljac != "exact" else 1e-9
    assert np.abs((s_schur - s_direct) / u).max() <= tol * ref
    assert np.abs((s_cg - s_direct) / u).max() <= max(tol, 1e-10) * ref
    # the correction solves J s = -f
    J = md.full_jacobian(p, U, eh, w.dt, 1.0, 0.0)
    resid = J @ (s_schur / u).ravel() + (f / u).ravel()
    assert np.abs(resid).max() <= 1e-11 * np.abs(f / u).max()


def test_schur_matrix_is_symmetric_positive_definite():
    """With D lagged the Schur matrix S = D - L M^-1 U is symmetric with positive face
    couplings and a positive local diagonal, so CG (Sec. 3.2.1) applies."""
    w = inputs.lognormal_hhe((4, 5, 6), box=150 * KPC, nsrc=3, dt=5e12)
    w.theta = 1.0
    p = oracle_problem(w)
    st = w.state()
    new, _ = sv.implicit_step(p, st, w.dt, 1.0, 0.0, 1e-9)
    U = md.state_to_U(p, new)
    g = md.build_g(p, U, new["e"], w.dt, 1.0, 0.0)
    f = md.residual(p, U, g, new["e"], w.dt, 1.0, 0.0)
    S, rhs, _, _ = sv.schur_system(p, U, f, new["e"], w.dt, 1.0, 0.0)
    Sd = S.toarray()
    assert np.array_equal(Sd, Sd.T)
    off = Sd - np.diag(np.diag(Sd))
    assert np.all(off <= 0)
    assert np.all(np.diag(Sd) + off.sum(axis=1) > 0)       # strictly diagonally dominant
    assert np.linalg.eigvalsh(Sd).min() > 0


def test_newton_linear_solvers_agree_and_conserve_elements():
    """The three exact linear solves reach the same root of f(U) = 0; species stay within
    their element totals (n_HI + n_HII = n_H, He likewise) cell by cell."""
    w = inputs.lognormal_hhe((6, 7, 8), box=200 * KPC, nsrc=3, dt=5e12)
    w.theta = 1.0
    p = oracle_problem(w, u_E=1e-18)
    st = w.state()
    outs = {}
    for lin in ("direct", "schur_direct", "schur_cg"):
        new, stats = sv.implicit_step(p, st, w.dt, 1.0, 0.0, 1e-12, linear=lin)
        assert stats["converged"], (lin, stats["res_history"])
        outs[lin] = new
    ref = outs["direct"]
    for lin in ("schur_direct", "schur_cg"):
        for key in ("E", "e", "n"):
            d = np.abs(outs[lin][key] - ref[key]).max() / np.abs(ref[key]).max()
            assert d < 1e-11, (lin, key, d)
    nHe = p.y_he * p.nH
    nHI, nHeI, nHeII = ref["n"]
    assert np.all(nHI > 0) and np.all(nHI < p.nH)
    assert np.all(nHeI > 0) and np.all(nHeII > 0) and np.all(nHeI + nHeII < nHe)


def test_newton_with_dD_dE_reaches_the_same_root():
    """Keeping dD/dE (Sec. 3.2.1) changes only the path: both Newton matrices reach the same
    root of f(U) = 0 where the radiation free-streams (small box, ionised bubbles)."""
    w = inputs.lognormal_hhe((10, 11, 12), box=50 * KPC, nsrc=3, dt=5e12)
    w.theta = 1.0
    st = w.state()
    p0 = oracle_problem(w, u_E=1e-17)
    st1, _ = sv.implicit_step(p0, st, w.dt, 1.0, 0.0, 1e-10, linear="direct")   # bubbles form
    out, its = {}, {}
    for lj in ("lagged", "E", "exact"):
        p = oracle_problem(w, u_E=1e-17, limiter_jacobian=lj)
        out[lj], stats = sv.implicit_step(p, st1, w.dt, 1.0, 0.0, 1e-11, linear="direct")
        assert stats["converged"], (lj, stats["res_history"])
        its[lj] = stats["res_history"]
    for lj in ("E", "exact"):
        for key in ("E", "e", "n"):
            d = np.abs(out[lj][key] - out["lagged"][key]).max() / np.abs(out["lagged"][key]).max()
            assert d < 1e-9, (lj, key, d)
    # the exact Newton matrix converges quadratically: the last residual ratio is tiny
    h = its["exact"]
    assert h[-1] / h[-2] < 1e-2, h


def test_rms_norm_definition():
    """Eq. rmsnorm: ||v|| = ||v||_2 / sqrt(N (N_s + 2)) over scaled components."""
    p = oracle_problem(inputs.lognormal_hhe((2, 2, 3), nsrc=1), u_e=2.0, u_n=4.0, u_E=8.0)
    f = np.ones((p.nv, p.N)) * p.scales()[:, None]
    assert abs(md.rms_norm(p, f) - 1.0) < 1e-15
    f[0, 0] = 0.0
    assert abs(md.rms_norm(p, f) - np.sqrt((p.nv * p.N - 1) / (p.nv * p.N))) < 1e-15


def test_explicit_predictor_is_explicit_euler():
    """Eq. explicit_predictor read as U^n - dt L(U^n) where no positivity cap binds."""
    w = inputs.lognormal_hhe((3, 4, 5), box=200 * KPC, nsrc=2, dt=1e9)
    p = oracle_problem(w)
    st = w.state()
    Un = md.state_to_U(p, st)
    L = md.full_operator(p, Un, st["e"], 1.0, 0.0)
    U0 = sv.explicit_predictor(p, Un, st["e"], w.dt, 1.0, 0.0)
    cap = sv.step_caps(p, Un, st["e"], -w.dt * L)
    free = cap == 1.0
    assert free.sum() > p.N // 2
    np.testing.assert_allclose(U0[:, free], (Un - w.dt * L)[:, free], rtol=1e-15)


@pytest.mark.parametrize("ns_case", ["h", "hhe"])
def test_step_caps_is_the_largest_feasible_fraction(ns_case):
    """The positivity cap (reading of the bounds limiter) is the largest fraction lam <= 1 of the
    step for which every bounded quantity keeps at least (1 - tau) of its distance to its
    bound.  Checked per cell by bisection on the stepped state itself: e = e^n + e_c, E and the
    species, with n_HII, n_HeIII derived from the stepped independent species, so the mapping
    of a step onto the derived species is pinned as well."""
    if ns_case == "h":
        w = inputs.uniform_h(4, shape=(3, 4, 5), box=60 * KPC, dt=3e12, nsteps=1, E0=1e-19)
    else:
        w = inputs.lognormal_hhe((3, 4, 5), box=200 * KPC, nsrc=2, dt=5e12, nsteps=1, seed=7)
    p = oracle_problem(w)
    st = w.state()
    U = md.state_to_U(p, st)
    eh = np.asarray(st["e"], dtype=np.float64).ravel()
    nH = p.nH.ravel()
    nHe = p.y_he * nH
    # cells at the species bounds: fully neutral (n_HII = 0), fully ionised (n_HI = 0), and for
    # helium n_HeIII = 0, n_HeI = 0, n_HeII = 0
    k = np.arange(p.N) % 6
    U[1, k == 0] = nH[k == 0]
    U[1, k == 1] = 0.0
    if p.ns == 3:
        U[3, k == 2] = nHe[k == 2] - U[2, k == 2]
        U[2, k == 3] = 0.0
        U[3, k == 4] = 0.0
    rng = np.random.default_rng(11)
    # steps of random sign over eight decades of each quantity's scale, so that every bound,
    # and every pair of species changes of similar size, binds somewhere
    tot = np.vstack([np.abs(eh)] + [nH] + [nHe] * (p.ns - 1) + [np.abs(U[1 + p.ns])])
    S = rng.uniform(-1.0, 1.0, size=U.shape) * tot * 10.0 ** rng.uniform(-8.0, 0.5, size=U.shape)
    cap = sv.step_caps(p, U, eh, S)

    def quantities(V, c):
        e = eh[c] + V[0]
        E = V[1 + p.ns]
        if p.ns == 1:
            nHI, nHeI, nHeII = V[1], 0.0, 0.0
        else:
            nHI, nHeI, nHeII = V[1], V[2], V[3]
        q = [(e, 0.0), (E, 0.0), (nHI, 1e-13 * nH[c]), (nH[c] - nHI, 1e-13 * nH[c])]
        if p.ns == 3:
            q += [(nHeI, 1e-13 * nHe[c]), (nHeII, 1e-13 * nHe[c]),
                  (nHe[c] - nHeI - nHeII, 1e-13 * nHe[c])]
        return q

    def feasible(c, lam):
        before = quantities(U[:, c], c)
        after = quantities(U[:, c] + lam * S[:, c], c)
        for (q0, tiny), (q1, _) in zip(before, after):
            # keep (1 - tau) of the distance q0 + tiny, up to the rounding of the stepped
            # quantity (a derived species carries that of its element total, 1e13 tiny)
            slack = 1e-15 * max(abs(q0), abs(q1), 1e13 * tiny)
            if q1 + tiny < (1.0 - p.tau) * (q0 + tiny) - slack:
                return False
        return True

    # a binding derived species near zero has a distance of order tiny, which the rounding
    # of its element total blurs at the 1e-3 level: the margin on both sides is 5%
    bound = 0
    for c in range(p.N):
        assert 0.0 <= cap[c] <= 1.0
        assert feasible(c, cap[c] * 0.95)
        if cap[c] < 1.0:
            assert not feasible(c, cap[c] * 1.05), (c, cap[c])
            bound += 1
    assert bound > 0


def test_backward_euler_block_of_cooling_gas_turns_singular():
    """Where radiative cooling falls with temperature, dL_e/de < 0 and the backward-Euler
    block M = I + theta dt dL/dx of eq. jacobian_submatrices passes through a singular matrix
    at a finite dt (det M changes sign).  One cell of photoionised H + He at z = 8.5, 10 times
    the mean comoving density (1331 times that, proper), 2e5 K, x_HI = 1e-3: M is regular at
    dt = 1e10 and 1e11 s and has changed the sign of its determinant by 1e12 s.  Steps longer
    than that cell's cooling time therefore cross a singular local elimination, which the
    cosmological configuration's adaptive steps of up to 1.4e14 s meet."""
    w = inputs.lognormal_hhe((1, 1, 1), box=inputs.MPC / 512, seed=0, nsrc=0)
    w.theta = 1.0
    w.u_E = 1e-14
    nH = 1e-2
    w.nH = np.full((1, 1, 1), nH)
    p = oracle_problem(w)
    a = 1.0 / 9.5
    H0 = 70e5 / inputs.MPC
    adot = a * H0 * np.sqrt(0.3 / a ** 3 + 0.7)
    y = w.y_he
    n = np.array([1e-3 * nH, 1e-3 * y * nH, 1e-2 * y * nH])
    ne = (nH - n[0]) + n[2] + 2.0 * (y * nH - n[1] - n[2])
    ntot = nH + y * nH + ne
    e = cl.K_BOLTZ * 2e5 * ntot / ((cl.GAMMA - 1.0) * cl.mass_density(nH, y * nH))
    U = np.concatenate([[0.0], n, [1e-14]]).reshape(-1, 1)
    dets = [np.linalg.det(md.local_blocks(p, U, np.array([e]), dt, a, adot)[0][0])
            for dt in (1e10, 1e11, 1e12, 1e13)]
    assert dets[0] > 0 and dets[1] > 0, dets
    assert dets[2] < 0 and dets[3] < 0, dets
