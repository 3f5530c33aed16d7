"""Seeded synthetic workloads for the implicit radiation / ionization step.

This module only draws inputs: grids, densities, initial states, point-source lists and the
per-run settings.  It holds none of the method's arithmetic and imports neither the solver
library nor the oracle; both sides consume what it returns.  The one conversion it does is the
initial condition's own definition: the gas energy of a gas at temperature T0 and the given
ionisation state (ideal gas, gamma = 5/3, as the workload is specified by T0).

Workload recipes (the paper's test problems are idealised set-ups, not datasets):

* ``uniform_h``      hydrogen only, uniform n_H, one central source split over the 8 cells
                     around the centre (odd sizes: the centre cell); monochromatic 13.6 eV.
* ``lognormal_hhe``  hydrogen + helium (Y = 0.24), lognormal n_H = nbar exp(s g - s^2 / 2)
                     with g a unit-variance Gaussian random field of power spectrum
                     P(k) ~ k^-2 (white noise filtered by k^-1 in Fourier space, k = 0
                     removed), point sources at uniformly drawn cells with lognormal photon
                     rates (median L50, log-sigma 1); T_B = 1e5 K blackbody spectrum.
"""
from dataclasses import dataclass, field

import numpy as np

MPC = 3.0857e24      # cm
KPC = 3.0857e21      # cm
_KB = 1.380649e-16   # erg/K   (initial-condition conversion only)
_MH = 1.67262192e-24 # g
_EV = 1.602176634e-12


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    dx: float                   # comoving cell width, cm
    ns: int                     # 1: H; 3: H + He
    y_he: float                 # n_He / n_H
    nH: np.ndarray              # (nz, ny, nx)
    E: np.ndarray               # (nz, ny, nx) erg / cm^3
    e: np.ndarray               # (nz, ny, nx) erg / g
    n: np.ndarray               # (ns, nz, ny, nx) independent species HI[, HeI, HeII]
    src_ijk: np.ndarray         # (nsrc, 3) cell indices (i, j, k)
    src_rate: np.ndarray        # (nsrc,) photons / s
    spectrum: tuple             # ("mono", photon energy erg) or ("blackbody", T_B)
    dt: float
    nsteps: int
    a: float = 1.0
    adot: float = 0.0
    newton_tol: float = 1e-8
    lin_tol: float = 1e-10
    theta: float = 0.51
    u_e: float = 1.0
    u_n: float = 1.0
    u_E: float = 1.0
    bc: tuple = ("zero_flux",) * 6
    bc_value: tuple = (0.0,) * 6  # E on Dirichlet faces, erg cm^-3
    meta: dict = field(default_factory=dict)
    schedule: list = None       # per step (dt, a, adot), cosmological runs
    model: str = "ionization"   # "ionization" (species) or "lte" (ns = 0, constant opacities)
    kappa_total: float = 0.0    # cm^-1 (LTE)
    kappa_planck: float = 0.0   # cm^-1 (LTE)
    mu: float = 0.6             # mean particle mass / m_H (LTE temperature)

    @property
    def N(self):
        return self.nx * self.ny * self.nz

    def state(self):
        """Flat copies (x fastest) of the initial state: dict(E, e, n)."""
        return dict(E=self.E.ravel().copy(), e=self.e.ravel().copy(),
                    n=self.n.reshape(self.ns, self.N).copy())


def _gas_energy(T0, nH, nHe, nHII, nHeII, nHeIII):
    """Specific energy of an ideal gas (gamma = 5/3) at T0 with the given ionisation."""
    ne = nHII + nHeII + 2.0 * nHeIII
    ntot = nH + nHe + ne
    rho = _MH * (nH + 4.0 * nHe)
    return 1.5 * _KB * T0 * ntot / rho


def gaussian_random_field(shape, seed, slope=-2.0):
    """Unit-variance Gaussian field with P(k) ~ k^slope (k = 0 mode removed)."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(shape)
    kz = np.fft.fftfreq(shape[0])[:, None, None]
    ky = np.fft.fftfreq(shape[1])[None, :, None]
    kx = np.fft.rfftfreq(shape[2])[None, None, :]
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(k)
    nz = k > 0
    amp[nz] = k[nz] ** (slope / 2.0)
    g = np.fft.irfftn(np.fft.rfftn(w) * amp, s=shape, axes=(0, 1, 2))
    g -= g.mean()
    sd = g.std()
    return g / sd if sd > 0 else g        # a single cell has no k > 0 mode


def uniform_h(n=32, box=1.0 * MPC, nH=1e-3, T0=100.0, x0=1e-4, E0=1e-20, ndot=5e48,
              dt=1e12, nsteps=5, newton_tol=1e-8, lin_tol=1e-10, shape=None, name=None,
              bc=("zero_flux",) * 6, source="centre"):
    """Hydrogen-only uniform medium with a central source (the 32^3, 1 Mpc benchmark), or with
    the source in the corner cell (0, 0, 0) (source = "corner", the HII-region test)."""
    nz, ny, nx = shape if shape is not None else (n, n, n)
    dx = box / nx
    nHf = np.full((nz, ny, nx), nH)
    nHII = x0 * nHf
    n_sp = (nHf - nHII)[None]
    z = np.zeros_like(nHf)
    e = _gas_energy(T0, nHf, z, nHII, z, z)
    # centre: the 8 cells around it for even sizes, the centre cell for odd sizes
    if source == "corner":
        cs = [[0], [0], [0]]
    else:
        cs = [[m // 2 - 1, m // 2] if m % 2 == 0 else [m // 2] for m in (nx, ny, nz)]
    ijk = np.array([(i, j, k) for k in cs[2] for j in cs[1] for i in cs[0]])
    rate = np.full(len(ijk), ndot / len(ijk))
    return Workload(name=name or f"uniform_h_{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=dx,
                    ns=1, y_he=0.0, nH=nHf, E=np.full_like(nHf, E0), e=e, n=n_sp,
                    src_ijk=ijk, src_rate=rate, spectrum=("mono", 13.6 * _EV), dt=dt,
                    nsteps=nsteps, newton_tol=newton_tol, lin_tol=lin_tol,
                    u_e=float(e.mean()), u_n=nH, u_E=E0, bc=tuple(bc))


def lognormal_hhe(shape=(128, 128, 128), box=1.0 * MPC, seed=0, nbar=1e-3, sigma_ln=1.0,
                  nsrc=16, L50=1e49, Y=0.24, T0=100.0, x0=1e-4, E0=1e-20, T_B=1e5, dt=5e12,
                  nsteps=20, newton_tol=1e-8, lin_tol=1e-10, name=None,
                  bc=("zero_flux",) * 6, clustered=False):
    """Hydrogen + helium lognormal medium with seeded point sources (128^3 / 256^3 runs);
    clustered sources sit in cells drawn with probability proportional to n_H^2."""
    nz, ny, nx = shape
    dx = box / nx
    g = gaussian_random_field(shape, seed)
    nH = nbar * np.exp(sigma_ln * g - 0.5 * sigma_ln ** 2)
    y_he = Y / (4.0 * (1.0 - Y))
    nHe = y_he * nH
    nHII = x0 * nH
    nHeII = x0 * nHe
    nHeIII = 1e-4 * x0 * nHe
    nHI = nH - nHII
    nHeI = nHe - nHeII - nHeIII
    e = _gas_energy(T0, nH, nHe, nHII, nHeII, nHeIII)
    rng = np.random.default_rng(seed + 7919)
    if clustered:
        w2 = (nH * nH).ravel()
        flat = rng.choice(nH.size, size=nsrc, replace=False, p=w2 / w2.sum())
        kk, jj, ii = np.unravel_index(flat, (nz, ny, nx))
        ijk = np.stack([ii, jj, kk], axis=1)
    else:
        ijk = np.stack([rng.integers(0, nx, nsrc), rng.integers(0, ny, nsrc),
                        rng.integers(0, nz, nsrc)], axis=1)
    rate = L50 * np.exp(rng.standard_normal(nsrc))
    return Workload(name=name or f"lognormal_hhe_{nx}x{ny}x{nz}_s{seed}", nx=nx, ny=ny, nz=nz,
                    dx=dx, ns=3, y_he=y_he, nH=nH, E=np.full_like(nH, E0), e=e,
                    n=np.stack([nHI, nHeI, nHeII]), src_ijk=ijk, src_rate=rate,
                    spectrum=("blackbody", T_B), dt=dt, nsteps=nsteps, newton_tol=newton_tol,
                    lin_tol=lin_tol, u_e=float(e.mean()), u_n=float(nH.mean()), u_E=E0,
                    bc=tuple(bc))


# the named benchmark workloads ----------------------------------------------------------------

def config_uniform_32():
    """Plain FP64 method: 32^3, 1 Mpc, H only, n_H = 1e-3, T0 = 100 K, x_HII = 1e-4, one
    central 5e48 s^-1 source at 13.6 eV, zero-flux boundaries, a = 1, 5 steps of 1e12 s.
    theta = 1: the set-up leaves theta open, and with c kappa dt = 189 in the neutral gas the
    theta = 0.51 step has no positive solution ((1 - theta) c kappa dt > 1 drives E below 0)."""
    w = uniform_h(32, name="uniform_h_32")
    w.theta = 1.0
    return w


# Radiation scaling u_E of the source-driven lognormal runs: a round number of the order of the
# energy density a median source (1e49 photons/s of mean energy ~47 eV) keeps one 3.9 kpc cell
# away, L <h nu> / (c dx^2) ~ 1.1e-16 erg/cm^3, so that scaled E is O(1-10) where the sources
# act (the 1e-20 ambient floor would put it at 1e5 there).
U_E_SOURCES = 1e-16


def config_lognormal(n=128, nsrc=16, seed=0, box=1.0 * MPC):
    """H + He lognormal medium (sigma_ln = 1, P(k) ~ k^-2, mean n_H = 1e-3), lognormal point
    sources (median 1e49 s^-1), 20 steps of 5e12 s, theta = 1; 128^3 with 16 sources or 256^3
    with 64 in a 1 Mpc box (sub-boxes keep the 256^3 cell size with box = n / 256 Mpc)."""
    w = lognormal_hhe((n, n, n), box=box, seed=seed, nsrc=nsrc, name=f"lognormal_hhe_{n}")
    w.theta = 1.0
    w.u_E = U_E_SOURCES
    return w


# flat Lambda-CDM expansion history (the cosmological configuration) -----------------------------

H0_KMS_MPC = 70.0       # km/s/Mpc
OMEGA_M = 0.3


def _h0():
    return H0_KMS_MPC * 1e5 / MPC                       # 1/s


def flat_lcdm_a(t, omega_m=OMEGA_M):
    """Scale factor of a flat matter + Lambda universe at cosmic time t (s):
    a = (Om / OL)^(1/3) sinh(3/2 sqrt(OL) H0 t)^(2/3)."""
    ol = 1.0 - omega_m
    return (omega_m / ol) ** (1.0 / 3.0) * np.sinh(1.5 * np.sqrt(ol) * _h0() * np.asarray(t)) ** (2.0 / 3.0)


def flat_lcdm_t(a, omega_m=OMEGA_M):
    """Inverse of flat_lcdm_a."""
    ol = 1.0 - omega_m
    return np.arcsinh((np.asarray(a) / (omega_m / ol) ** (1.0 / 3.0)) ** 1.5) / (1.5 * np.sqrt(ol) * _h0())


def flat_lcdm_adot(a, omega_m=OMEGA_M):
    """da/dt = a H(a) = a H0 sqrt(Om a^-3 + OL)."""
    a = np.asarray(a)
    return a * _h0() * np.sqrt(omega_m / a ** 3 + (1.0 - omega_m))


# Radiation scaling of the cosmological configuration.  Its adaptive steps reach 1.4e14 s, where
# c kappa dt in the dense neutral cells is of order 1e7: the radiation row of f is then a
# difference of terms 1e7 times E, whose FP64 rounding the RMS tolerance must not have to
# resolve.  With u_E = 1e-16 (the static runs' value) those steps stalled at ||f|| = 1e-8 to
# 5e-7 after 40 Newton iterations; with 1e-14 each interval after the first takes one step.
U_E_COSMO = 1e-14


def config_cosmo(n=512, nsrc=256, seed=0, box=1.0 * MPC, z0=10.0, z1=6.0, nsteps=100):
    """The cosmological configuration: H + He lognormal medium with sigma_ln = 1.5 (comoving
    mean n_H = 1e-3), 256 lognormal sources in cells drawn with probability ~ n_H^2, theta = 1,
    expansion from z = 10 to z = 6 in equal steps of cosmic time.  ``schedule`` holds (dt, a,
    adot) of each step, a and adot taken at the middle of the step."""
    w = lognormal_hhe((n, n, n), box=box, seed=seed, nsrc=nsrc, sigma_ln=1.5, clustered=True,
                      nsteps=nsteps, name=f"cosmo_hhe_{n}", dt=1.0)
    w.theta = 1.0
    w.u_E = U_E_COSMO
    t0, t1 = flat_lcdm_t(1.0 / (1.0 + z0)), flat_lcdm_t(1.0 / (1.0 + z1))
    dt = (t1 - t0) / nsteps
    w.dt = float(dt)
    mids = t0 + (np.arange(nsteps) + 0.5) * dt
    a = flat_lcdm_a(mids)
    w.schedule = [(float(dt), float(ai), float(flat_lcdm_adot(ai))) for ai in a]
    return w


# the cosmological I-front (the Shapiro-Giroux set-up) -------------------------------------------

# (q0, z_i) -> (H0 in 100 km/s/Mpc, Omega_m, initial baryon density g cm^-3, initial proper box kpc)
SG_CASES = {(0.5, 4.0): (0.5, 1.0, 1.175e-28, 80.0), (0.05, 4.0): (1.0, 0.1, 2.35e-28, 60.0),
            (0.5, 10.0): (0.5, 1.0, 1.175e-28, 36.0), (0.05, 10.0): (1.0, 0.1, 2.35e-28, 27.0)}


def config_sg(n=32, q0=0.5, z_i=4.0, ndot=5e48, T=1e4, E0_proper=1e-35):
    """Hydrogen of uniform comoving density around a 13.6 eV source in a matter-only universe
    of deceleration parameter q0, from redshift z_i: the four parameter sets of the
    cosmological radiative-ionization test (initial box and baryon density as listed there),
    T = 1e4 K held, neutral gas (x_HII = 0), E = 1e-35 erg cm^-3 proper.  The source sits in
    the corner cell of one octant (reflecting faces), which therefore emits ndot / 8.  Scale
    factors a = 1 / (1 + z); densities and E are comoving (proper times a^3); dx is comoving."""
    h, om, rho_i, box_kpc = SG_CASES[(q0, z_i)]
    a_i = 1.0 / (1.0 + z_i)
    nH_i = rho_i / _MH                                   # proper, hydrogen only
    w = uniform_h(n, box=box_kpc * KPC / a_i, nH=nH_i * a_i ** 3, T0=T, x0=0.0,
                  E0=E0_proper * a_i ** 3, ndot=ndot / 8.0, source="corner",
                  name=f"sg_q{q0}_z{z_i}_{n}")
    w.theta = 1.0
    w.u_E = 1e-20
    w.meta.update(q0=q0, z_i=z_i, a_i=a_i, H0=h * 100e5 / MPC, omega_m=om, nH_i=nH_i,
                  ndot=ndot)
    return w


def matter_only_adot(a, H0, omega_m):
    """da/dt of a universe with matter and curvature only: a H0 sqrt(Om a^-3 + (1 - Om) a^-2)."""
    a = np.asarray(a, dtype=np.float64)
    return a * H0 * np.sqrt(omega_m / a ** 3 + (1.0 - omega_m) / a ** 2)


# LTE coupling: matter-radiation equilibration (the Turner-Stone set-up) ---------------------------

def lte_uniform(e_vol, n=4, rho=1e-7, E0=1e12, kappa=4e-8, mu=0.6, box=1.0, dt=1e-12, nsteps=50,
                bc=("periodic",) * 6, E_perturb=0.0, seed=0):
    """A box of uniform LTE gas (eq. LTE_coupling) with gas energy density e_vol (erg cm^-3),
    density rho, radiation energy density E0 and one opacity for both means; E_perturb adds a
    seeded relative perturbation to E so that diffusion takes part.  Box in cm."""
    nH = np.full((n, n, n), rho / _MH)
    e = np.full_like(nH, e_vol / rho)
    E = np.full_like(nH, E0)
    if E_perturb:
        E = E * (1.0 + E_perturb * np.random.default_rng(seed).standard_normal(E.shape))
    return Workload(name=f"lte_{n}", nx=n, ny=n, nz=n, dx=box / n, ns=0, y_he=0.0, nH=nH,
                    E=E, e=e, n=np.zeros((0, n, n, n)), src_ijk=np.zeros((0, 3), dtype=np.int64),
                    src_rate=np.zeros(0), spectrum=("mono", 13.6 * _EV), dt=dt, nsteps=nsteps,
                    theta=1.0, u_e=float(e.mean()), u_n=1.0, u_E=float(E0), bc=tuple(bc),
                    model="lte", kappa_total=kappa, kappa_planck=kappa, mu=mu)

