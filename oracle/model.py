"""Oracle model: theta-scheme operators, nonlinear residual, analytic Jacobian, RMS norm.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Everything is plain vectorised numpy over cells, FP64.  Arrays are flat over cells with the
index  i + nx (j + ny k)  (x fastest).  The unknown vector of one cell is
U = (e_c, n_1 .. n_Ns, E)  (Sec. 3.2, above eq. nonlinear_residual), with the independent
species n = (n_HI) for hydrogen only and n = (n_HI, n_HeI, n_HeII) for hydrogen + helium;
n_HII, n_HeIII and n_e follow from element conservation.

Readings of the paper made here (each also listed in the design notes):
* L_n (eq. mLn) is written out species by species with photoionisation, collisional
  ionisation and case-B recombination; L_e (eq. mLe) with photoheating G and cooling Lambda.
* The "c k E" of eq. mLE is read as c kappa E (as in eq. cons_radiation).
* Proper densities enter the two-body and photo terms: a factor 1/a^3 (eq. proper_vars);
  the diffusion operator is (1/a^2) div(D grad E) with R = |grad E| / (a E).  At a = 1 this
  is exactly eq. RT-cons_radiation.
* The limiter's R_i = |d_i E| / E (eq. limiter) is discretised per face as
  |E_b - E_a| / (a dx (E_a + E_b)/2), floored at 1 / (a L) with L the largest extent of
  the grid; kappa at a face is the mean of the two cells' kappa.  ``limiter = False`` gives
  D = c / (3 max(kappa, kappa_floor)).
* The Newton matrix either lags D entirely (``limiter_jacobian = "lagged"``: the Schur matrix is
  symmetric, as CG needs) or, as Sec. 3.2.1 states, keeps dD/dE and lags only the opacity
  (``"E"``: a non-symmetric Schur matrix), or keeps both dD/dE and the opacity's species
  dependence (``"exact"``: the true Jacobian of f; its Schur complement is still a 7-point
  operator in E because the cell-local blocks are eliminated cell by cell).
"""
from dataclasses import dataclass, field

import numpy as np
from scipy import sparse

from . import closure as cl

BC_ZERO_FLUX = "zero_flux"
BC_PERIODIC = "periodic"
BC_DIRICHLET = "dirichlet"


@dataclass
class Problem:
    """Grid, boundary conditions, closure and solver parameters of one implicit solve."""
    nx: int
    ny: int
    nz: int
    dx: float                          # comoving cell width, cm (cubic cells)
    ns: int                            # independent species: 1 (H) or 3 (H + He)
    nH: np.ndarray                     # comoving hydrogen number density per cell
    src: np.ndarray                    # 4 pi eta per cell, erg cm^-3 s^-1 (comoving)
    grey: dict                         # sk, pgam, ph arrays over (HI, HeI, HeII)
    y_he: float = 0.0                  # n_He / n_H
    bc: tuple = (BC_ZERO_FLUX,) * 6    # faces x-, x+, y-, y+, z-, z+
    bc_value: tuple = (0.0,) * 6       # E on Dirichlet faces, erg cm^-3
    theta: float = 0.51                # Sec. 3.2, below eq. radiation_simplified
    m_grey: int = 1                    # m of eq. cons_radiation
    isothermal: bool = False           # fixed temperature, e_c == 0 (Sec. 4.5 test setup)
    limiter: bool = True               # eq. limiter on/off
    kappa_floor: float = 1e-40         # cm^-1, only used without the limiter
    u_e: float = 1.0                   # scalings of eq. scalings (supplied per problem)
    u_n: float = 1.0
    u_E: float = 1.0
    tau: float = 0.99                  # fraction-to-boundary of the positivity limiter
    lam_min: float = 1.0 / 16.0         # smallest line-search parameter
    limiter_jacobian: str = "lagged"   # "lagged": D frozen in J; "E": dD/dE kept, kappa lagged;
                                       # "exact": dD/dE and dD/dkappa dkappa/dn kept
    growth_max: float = 1e3            # watchdog: a full step may raise ||f|| up to this factor
    watchdog: int = 3                  # ... for at most this many steps without a new best ||f||
    rates: object = field(default=None)
    # LTE coupling (eq. LTE_coupling): no species (ns = 0), constant total and Planck-mean
    # opacities, temperature from e with a fixed mean particle mass mu m_H
    model: str = "ionization"          # "ionization" (non-LTE, Sec. 2.1) or "lte"
    kappa_total: float = 0.0           # cm^-1
    kappa_planck: float = 0.0          # cm^-1
    mu: float = 0.6

    def __post_init__(self):
        if self.rates is None:
            self.rates = cl.RateTable()
        self.nH = np.ascontiguousarray(self.nH, dtype=np.float64).ravel()
        self.src = np.ascontiguousarray(self.src, dtype=np.float64).ravel()
        if self.ns == 1 and self.y_he != 0.0:
            raise ValueError("hydrogen-only runs have y_he = 0")
        if (self.model == "lte") != (self.ns == 0):
            raise ValueError("the LTE model has no species (ns = 0), the ionization model 1 or 3")
        for lo, hi in ((0, 1), (2, 3), (4, 5)):
            if (self.bc[lo] == BC_PERIODIC) != (self.bc[hi] == BC_PERIODIC):
                raise ValueError("periodic boundaries come in pairs")

    @property
    def N(self):
        return self.nx * self.ny * self.nz

    @property
    def nv(self):
        return self.ns + 2

    def scales(self):
        return np.array([self.u_e] + [self.u_n] * self.ns + [self.u_E])

    def species_full(self, n):
        """(nHI, nHeI, nHeII) with zeros for absent helium."""
        z = np.zeros_like(n[0])
        if self.ns == 1:
            return n[0], z, z
        return n[0], n[1], n[2]


# --------------------------------------------------------------------------------------------
# neighbours and boundary conditions

def neighbor_table(p):
    """For each cell and direction (-x, +x, -y, +y, -z, +z): neighbour flat index and whether
    the face carries flux (False on zero-flux boundary faces)."""
    k, j, i = np.meshgrid(np.arange(p.nz), np.arange(p.ny), np.arange(p.nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    nb = np.empty((6, p.N), dtype=np.int64)
    valid = np.ones((6, p.N), dtype=bool)
    dims = (p.nx, p.ny, p.nz)
    coords = [i, j, k]
    for d in range(6):
        ax, step = d // 2, (-1 if d % 2 == 0 else 1)
        c = [i.copy(), j.copy(), k.copy()]
        c[ax] = coords[ax] + step
        out = (c[ax] < 0) | (c[ax] >= dims[ax])
        if p.bc[d] == BC_PERIODIC:
            c[ax] = np.mod(c[ax], dims[ax])
        else:
            valid[d] = ~out
            c[ax] = np.clip(c[ax], 0, dims[ax] - 1)
        nb[d] = c[0] + p.nx * (c[1] + p.ny * c[2])
    return nb, valid


# --------------------------------------------------------------------------------------------
# local (cell-wise) physics, eqs. mLe, mLn, mLE with their derivatives

def local_terms(p, ec, n, E, eh, nH, src, a, adot, T_fixed=None, want_jac=False):
    """Reaction operators of a set of cells (n_H and 4 pi eta given per cell) and, if
    ``want_jac``, their partial derivatives:
      L          [L_e, L_n1, ..] (eqs. mLe, mLn);  LE  local part of eq. mLE;  kappa, T
      dLx[a][b]  d(local operator a) / d(unknown b), a, b over (e_c, n_1, ..)
      dLxE[a]    d(local operator a) / dE
      dLEx[b]    d LE / d(unknown b);   dLEE  d LE / dE""" 
    if p.model == "lte":
        return _local_terms_lte(p, ec, E, eh, nH, src, a, adot, T_fixed, want_jac)
    ns = p.ns
    c = cl.C_LIGHT
    ia3 = 1.0 / a ** 3
    nHe = p.y_he * nH
    nHI, nHeI, nHeII = p.species_full(n)
    nHII, nHeIII, ne = cl.derived_species(nH, nHe, nHI, nHeI, nHeII)
    rho = cl.mass_density(nH, nHe)
    e = eh + ec
    ntot = nH + nHe + ne
    if p.isothermal:
        T = T_fixed
        dT_dec = np.zeros_like(e)
        dT_dne = np.zeros_like(e)
    else:
        T = cl.temperature(e, nH, nHe, ne)
        dT_dec = T / e                       # T is proportional to e
        dT_dne = -T / ntot                   # d n_tot = d n_e
    k, dk = p.rates(T)
    aHII, bHI, aHeII, bHeI, aHeIII, bHeII = (k[..., r] for r in range(6))
    C = (k[..., 6] * nHI + k[..., 7] * nHII + k[..., 8] * nHeI + k[..., 9] * nHeII
         + k[..., 10] * nHeIII)
    sk, pg, ph = p.grey["sk"], p.grey["pgam"], p.grey["ph"]

    # photoionisation rates Gamma_X = c pgam_X E_proper (eq. adaptive_spectrum)
    GHI, GHeI, GHeII = (c * pg[X] * E * ia3 for X in range(3))
    # two-body brackets B (rates times densities) of each species operator
    B = [bHI * nHI - aHII * nHII]
    A = [GHI * nHI]
    if ns == 3:
        B.append(bHeI * nHeI - aHeII * nHeII)
        B.append((bHeII + aHeII) * nHeII - bHeI * nHeI - aHeIII * nHeIII)
        A.append(GHeI * nHeI)
        A.append(GHeII * nHeII - GHeI * nHeI)
    Ln = [A[s] + ia3 * ne * B[s] for s in range(ns)]                     # eq. mLn

    heat_sum = ph[0] * nHI + ph[1] * nHeI + ph[2] * nHeII
    G = c * E * ia3 * heat_sum / rho
    Lam = ia3 * ne * C / rho
    if p.isothermal:
        Le = np.zeros_like(e)
    else:
        Le = 2.0 * (adot / a) * ec - G + Lam                             # eq. mLe
    kap = ia3 * (sk[0] * nHI + sk[1] * nHeI + sk[2] * nHeII)
    LE = p.m_grey * (adot / a) * E - src + c * kap * E                   # eq. mLE
    out = dict(L=[Le] + Ln, LE=LE, kappa=kap, T=T, ne=ne, rho=rho)
    if not want_jac:
        return out

    # ----- derivatives (eq. jacobian_submatrices) -----
    dne = [-1.0, -2.0, -1.0][:ns]             # d n_e / d (n_HI, n_HeI, n_HeII)
    # dB/dn at fixed T and dB/dT
    dBdn = [[bHI + aHII]]
    dBdT = [dk[..., 1] * nHI - dk[..., 0] * nHII]
    dAdn = [[GHI]]
    dAdE = [c * pg[0] * ia3 * nHI]
    if ns == 3:
        zero = np.zeros_like(e)
        dBdn = [[bHI + aHII, zero, zero],
                [zero, bHeI, -aHeII],
                [zero, -bHeI + aHeIII, bHeII + aHeII + aHeIII]]
        dBdT.append(dk[..., 3] * nHeI - dk[..., 2] * nHeII)
        dBdT.append((dk[..., 5] + dk[..., 2]) * nHeII - dk[..., 3] * nHeI
                    - dk[..., 4] * nHeIII)
        dAdn = [[GHI, zero, zero],
                [zero, GHeI, zero],
                [zero, -GHeI, GHeII]]
        dAdE.append(c * pg[1] * ia3 * nHeI)
        dAdE.append(c * ia3 * (pg[2] * nHeII - pg[1] * nHeI))
    dCdn = [k[..., 6] - k[..., 7], k[..., 8] - k[..., 10], k[..., 9] - k[..., 10]][:ns]
    dCdT = (dk[..., 6] * nHI + dk[..., 7] * nHII + dk[..., 8] * nHeI + dk[..., 9] * nHeII
            + dk[..., 10] * nHeIII)
    dTdn = [dT_dne * dne[j] for j in range(ns)]

    nm = ns + 1
    dLx = [[None] * nm for _ in range(nm)]
    dLxE = [None] * nm
    # energy row
    if p.isothermal:
        z = np.zeros_like(e)
        dLx[0][0] = z
        for j in range(ns):
            dLx[0][1 + j] = z
        dLxE[0] = z
    else:
        dLx[0][0] = 2.0 * adot / a + ia3 * ne * dCdT * dT_dec / rho
        for j in range(ns):
            dLx[0][1 + j] = (-c * E * ia3 * ph[j] / rho
                             + ia3 / rho * (dne[j] * C + ne * dCdn[j] + ne * dCdT * dTdn[j]))
        dLxE[0] = -c * ia3 * heat_sum / rho
    # species rows
    for s in range(ns):
        dLx[1 + s][0] = ia3 * ne * dBdT[s] * dT_dec
        for j in range(ns):
            dLx[1 + s][1 + j] = (dAdn[s][j]
                                 + ia3 * (dne[j] * B[s] + ne * dBdn[s][j] + ne * dBdT[s] * dTdn[j]))
        dLxE[1 + s] = dAdE[s]
    dLEx = [np.zeros_like(e)] + [c * ia3 * sk[j] * E for j in range(ns)]
    dLEE = p.m_grey * adot / a + c * kap
    out.update(dLx=dLx, dLxE=dLxE, dLEx=dLEx, dLEE=dLEE)
    return out


def _local_terms_lte(p, ec, E, eh, nH, src, a, adot, T_fixed, want_jac):
    """Local operators of the LTE model (eq. LTE_coupling): emission 4 pi eta = 4 kappa_P
    sigma_SB T^4, heating G = c kappa E / rho and cooling Lambda = 4 pi eta / rho, with
    T = (gamma - 1) mu m_H e / k_B.  L_e = 2 (adot/a) e_c - G + Lambda (eq. mLe with these
    terms) and the local part of L_E = m (adot/a) E - 4 pi eta_src + c kappa E - 4 pi eta
    (eq. mLE).  The opacities are used as given (no 1/a^3 factor)."""
    c = cl.C_LIGHT
    e = eh + ec
    rho = cl.M_H * nH * (1.0 + 4.0 * p.y_he)
    cT = (cl.GAMMA - 1.0) * p.mu * cl.M_H / cl.K_BOLTZ      # T = cT e
    if p.isothermal:
        T = T_fixed
        dT_dec = np.zeros_like(e)
    else:
        T = cT * e
        dT_dec = np.full_like(e, cT)
    kap = np.full_like(e, p.kappa_total)
    emis = 4.0 * p.kappa_planck * cl.SIGMA_SB * T ** 4                # 4 pi eta_LTE
    G = c * p.kappa_total * E / rho
    Lam = emis / rho
    Le = np.zeros_like(e) if p.isothermal else 2.0 * (adot / a) * ec - G + Lam
    LE = p.m_grey * (adot / a) * E - src + c * p.kappa_total * E - emis
    out = dict(L=[Le], LE=LE, kappa=kap, T=T, ne=np.zeros_like(e), rho=rho)
    if not want_jac:
        return out
    demis = 16.0 * p.kappa_planck * cl.SIGMA_SB * T ** 3 * dT_dec     # d(4 pi eta)/d e_c
    if p.isothermal:
        dLx = [[np.zeros_like(e)]]
        dLxE = [np.zeros_like(e)]
    else:
        dLx = [[2.0 * adot / a + demis / rho]]
        dLxE = [-c * p.kappa_total / rho]
    dLEx = [-demis]
    dLEE = p.m_grey * adot / a + c * p.kappa_total + 0.0 * e
    out.update(dLx=dLx, dLxE=dLxE, dLEx=dLEx, dLEE=dLEE)
    return out


# --------------------------------------------------------------------------------------------
# diffusion (eq. mDE with eq. limiter)

def face_coefficient(p, Ea, Eb, ka, kb, a, h=None):
    """D_face / (a^2 dx h) for a face between points a and b a distance h apart (default dx:
    two cells; dx/2: a cell and a Dirichlet boundary value), per unit time, 1/s.

    R is floored at 1 / (a L), L the largest comoving extent of the grid, so that D <= c a L
    where the radiation field is flat and the medium transparent (kappa = R = 0 leaves
    eq. limiter undefined).  Without the limiter D = c / (3 max(kappa, kappa_floor))."""
    h = p.dx if h is None else h
    kap = 0.5 * (ka + kb)
    c = cl.C_LIGHT
    if p.limiter:
        Ebar = 0.5 * (Ea + Eb)
        R_min = 1.0 / (a * max(p.nx, p.ny, p.nz) * p.dx)
        R = np.maximum(np.abs(Eb - Ea) / (a * h * Ebar), R_min)
        D = c * (2.0 * kap + R) / (6.0 * kap ** 2 + 3.0 * kap * R + R ** 2)   # eq. limiter
    else:
        D = c / (3.0 * np.maximum(kap, p.kappa_floor))
    return D / (a * a * p.dx * h)


def face_coefficient_derivatives(p, Ea, Eb, ka, kb, a, h=None):
    """(W, dW/dE_a, dW/dE_b) of ``face_coefficient`` with kappa held fixed (Sec. 3.2.1 lags
    only the opacity dependence of D).  dD/dR = -c R (4 kappa + R) / (6 kappa^2 + 3 kappa R +
    R^2)^2 and dR/dE_{a,b} = -/+ sign(E_b - E_a) / (a dx Ebar) - R / (2 Ebar); zero where R
    sits at its floor or without the limiter."""
    h = p.dx if h is None else h
    W = face_coefficient(p, Ea, Eb, ka, kb, a, h)
    if not p.limiter:
        z = np.zeros_like(W)
        return W, z, z
    kap = 0.5 * (ka + kb)
    c = cl.C_LIGHT
    Ebar = 0.5 * (Ea + Eb)
    R_min = 1.0 / (a * max(p.nx, p.ny, p.nz) * p.dx)
    Rraw = np.abs(Eb - Ea) / (a * h * Ebar)
    live = Rraw > R_min
    R = np.maximum(Rraw, R_min)
    den = 6.0 * kap ** 2 + 3.0 * kap * R + R ** 2
    dDdR = -c * R * (4.0 * kap + R) / den ** 2
    sgn = np.sign(Eb - Ea)
    dRa = -sgn / (a * h * Ebar) - R / (2.0 * Ebar)
    dRb = sgn / (a * h * Ebar) - R / (2.0 * Ebar)
    f = np.where(live, dDdR / (a * a * p.dx * h), 0.0)
    return W, f * dRa, f * dRb


def face_coefficient_kappa_derivative(p, Ea, Eb, ka, kb, a, h=None):
    """dW/dkappa_face of ``face_coefficient`` at fixed E: with the limiter
    dD/dkappa = -c (12 kappa^2 + 12 kappa R + R^2) / (6 kappa^2 + 3 kappa R + R^2)^2 (the
    quotient rule on eq. limiter), without it -c / (3 kappa^2) above the floor, else 0.  Each
    cell's kappa enters the face mean with weight 1/2."""
    h = p.dx if h is None else h
    kap = 0.5 * (ka + kb)
    c = cl.C_LIGHT
    if p.limiter:
        Ebar = 0.5 * (Ea + Eb)
        R_min = 1.0 / (a * max(p.nx, p.ny, p.nz) * p.dx)
        R = np.maximum(np.abs(Eb - Ea) / (a * h * Ebar), R_min)
        den = 6.0 * kap ** 2 + 3.0 * kap * R + R ** 2
        dD = -c * (12.0 * kap ** 2 + 12.0 * kap * R + R ** 2) / den ** 2
    else:
        dD = np.where(kap > p.kappa_floor, -c / (3.0 * np.maximum(kap, p.kappa_floor) ** 2), 0.0)
    return dD / (a * a * p.dx * h)


def dirichlet_faces(p):
    """[(d, mask, E_b)] for every Dirichlet face d (0..5 = x-, x+, y-, y+, z-, z+): the cells
    next to it and the boundary value.  The value sits on the boundary, half a cell from the
    cell centre."""
    if BC_DIRICHLET not in p.bc:
        return []
    k, j, i = np.meshgrid(np.arange(p.nz), np.arange(p.ny), np.arange(p.nx), indexing="ij")
    q = (i.ravel(), j.ravel(), k.ravel())
    dims = (p.nx, p.ny, p.nz)
    out = []
    for d in range(6):
        if p.bc[d] == BC_DIRICHLET:
            ax = d // 2
            m = q[ax] == (0 if d % 2 == 0 else dims[ax] - 1)
            out.append((d, m, float(p.bc_value[d])))
    return out


def diffusion_kappa_block(p, E, kap, a, dth, nbt):
    """d(dt theta * diffusion term of cell i) / d kappa_j for j = i (diag) and the flux-carrying
    neighbours (rows, cols, vals): face f between i and nb contributes
    dt theta (1/2) dW_f/dkappa_f (E_i - E_nb) to both."""
    nb, valid = nbt
    N = p.N
    cells = np.arange(N)
    diag = np.zeros(N)
    rows, cols, vals = [], [], []
    for d in range(6):
        m = valid[d]
        Enb, knb = E[nb[d]], kap[nb[d]]
        v = dth * 0.5 * face_coefficient_kappa_derivative(p, E, Enb, kap, knb, a) * (E - Enb)
        diag += np.where(m, v, 0.0)
        rows.append(cells[m]); cols.append(nb[d][m]); vals.append(v[m])
    for d, m, Eb in dirichlet_faces(p):
        # the boundary face's opacity is the cell's own (weight 1)
        v = dth * face_coefficient_kappa_derivative(p, E, Eb, kap, kap, a, 0.5 * p.dx) * (E - Eb)
        diag += np.where(m, v, 0.0)
    return diag, rows, cols, vals


def face_weights(p, E, kap, a, nbt=None):
    """W[d, cell] for the six faces of every cell (0 on zero-flux boundary faces)."""
    nb, valid = neighbor_table(p) if nbt is None else nbt
    W = np.zeros((6, p.N))
    for d in range(6):
        W[d] = np.where(valid[d], face_coefficient(p, E, E[nb[d]], kap, kap[nb[d]], a), 0.0)
    for d, m, Eb in dirichlet_faces(p):       # boundary faces: distance dx/2, kappa of the cell
        W[d] = np.where(m, face_coefficient(p, E, Eb, kap, kap, a, 0.5 * p.dx), W[d])
    return W


def diffusion_term(p, E, W, nbt=None):
    """-div(D grad E) / a^2 per unit time: sum over faces W (E_i - E_nb)."""
    nb, valid = neighbor_table(p) if nbt is None else nbt
    out = np.zeros(p.N)
    for d in range(6):
        out += np.where(valid[d], W[d] * (E - E[nb[d]]), 0.0)
    for d, m, Eb in dirichlet_faces(p):
        out += np.where(m, W[d] * (E - Eb), 0.0)
    return out


# --------------------------------------------------------------------------------------------
# full operator, g^n and residual (eqs. energy/chemistry/radiation_simplified, nonlinear_residual)

def full_operator(p, U, eh, a, adot, T_fixed=None, nbt=None, W=None, kap_faces=None):
    """L(U) for every unknown: (L_e, L_n.., D_E + L_E) stacked as (nv, N).  ``W`` freezes the
    face coefficients and ``kap_faces`` only the opacity inside them (used to check the two
    Newton matrices by finite differences)."""
    ns = p.ns
    ec, n, E = U[0], U[1:1 + ns], U[1 + ns]
    lt = local_terms(p, ec, n, E, eh, p.nH, p.src, a, adot, T_fixed)
    if W is None:
        W = face_weights(p, E, lt["kappa"] if kap_faces is None else kap_faces, a, nbt)
    Lfull = np.empty_like(U)
    for v in range(ns + 1):
        Lfull[v] = lt["L"][v]
    Lfull[1 + ns] = diffusion_term(p, E, W, nbt) + lt["LE"]
    return Lfull


def state_to_U(p, state):
    """Newton unknowns at t^n: (e_c^n = 0, n^n, E^n) (Sec. 3.1: e_c^n = 0)."""
    U = np.empty((p.nv, p.N))
    U[0] = 0.0
    U[1:1 + p.ns] = np.asarray(state["n"]).reshape(p.ns, p.N)
    U[1 + p.ns] = np.asarray(state["E"]).ravel()
    return U


def fixed_temperature(p, state):
    """Temperature of each cell of a state (e, n); isothermal runs hold it fixed."""
    eh = np.asarray(state["e"]).ravel()
    if p.model == "lte":
        return (cl.GAMMA - 1.0) * p.mu * cl.M_H / cl.K_BOLTZ * eh
    n = np.asarray(state["n"]).reshape(p.ns, p.N)
    nHI, nHeI, nHeII = p.species_full(n)
    nHe = p.y_he * p.nH
    _, _, ne = cl.derived_species(p.nH, nHe, nHI, nHeI, nHeII)
    return cl.temperature(eh, p.nH, nHe, ne)


def build_g(p, Un, eh, dt, a, adot, T_fixed=None, nbt=None):
    """g^n = U^n + dt (theta - 1) L(U^n), the right-hand sides of eqs. *_simplified."""
    return Un + dt * (p.theta - 1.0) * full_operator(p, Un, eh, a, adot, T_fixed, nbt)


def residual(p, U, g, eh, dt, a, adot, T_fixed=None, nbt=None, W=None, kap_faces=None):
    """f(U) = U + dt theta L(U) - g^n  (eq. nonlinear_residual)."""
    return U + dt * p.theta * full_operator(p, U, eh, a, adot, T_fixed, nbt, W, kap_faces) - g


def rms_norm(p, f):
    """Eq. rmsnorm over the scaled residual (eq. scalings): ||f/u||_2 / sqrt(N (Ns + 2))."""
    fs = f / p.scales()[:, None]
    return float(np.sqrt(np.sum(fs * fs) / (p.N * p.nv)))


# --------------------------------------------------------------------------------------------
# Newton matrix (eqs. jacobian_matrix, newton_system2, schur_components)

def local_blocks(p, U, eh, dt, a, adot, T_fixed=None):
    """Scaled cell-local blocks of J at U:  M (N, nm, nm), Ucol (N, nm), Lrow (N, nm),
    Dloc (N,), with nm = Ns + 1, all in the scaled unknowns of eq. scalings.  D_loc holds
    only the local part of D = I + dt theta J_EE; the diffusion part is ``face_weights``."""
    ns, nm = p.ns, p.ns + 1
    ec, n, E = U[0], U[1:1 + ns], U[1 + ns]
    lt = local_terms(p, ec, n, E, eh, p.nH, p.src, a, adot, T_fixed, want_jac=True)
    dth = dt * p.theta
    u = p.scales()
    uM, uE = u[:nm], u[nm]
    M = np.zeros((p.N, nm, nm))
    Ucol = np.zeros((p.N, nm))
    Lrow = np.zeros((p.N, nm))
    for r in range(nm):
        for s in range(nm):
            M[:, r, s] = (1.0 if r == s else 0.0) + dth * lt["dLx"][r][s] * uM[s] / uM[r]
        Ucol[:, r] = dth * lt["dLxE"][r] * uE / uM[r]
        Lrow[:, r] = dth * lt["dLEx"][r] * uM[r] / uE
    Dloc = 1.0 + dth * lt["dLEE"]
    return M, Ucol, Lrow, Dloc, lt


def diffusion_block(p, E, kap, a, dth, nbt):
    """The diffusion part of D = I + dt theta J_EE (eq. schur_components) as (diag, rows,
    cols, vals): with D lagged, face f adds dt theta W_f to the diagonal and -dt theta W_f to
    the neighbour column; with dD/dE kept (Sec. 3.2.1) the entries of row i are
    dt theta [W_f + dW_f/dE_i (E_i - E_nb)] and dt theta [-W_f + dW_f/dE_nb (E_i - E_nb)]."""
    nb, valid = nbt
    N = p.N
    cells = np.arange(N)
    diag = np.zeros(N)
    rows, cols, vals = [], [], []
    for d in range(6):
        m = valid[d]
        Enb, knb = E[nb[d]], kap[nb[d]]
        if p.limiter_jacobian in ("E", "exact"):
            W, dWi, dWn = face_coefficient_derivatives(p, E, Enb, kap, knb, a)
            dE = E - Enb
            di = W + dWi * dE
            off = -W + dWn * dE
        else:
            W = face_coefficient(p, E, Enb, kap, knb, a)
            di, off = W, -W
        diag += np.where(m, dth * di, 0.0)
        rows.append(cells[m]); cols.append(nb[d][m]); vals.append(dth * off[m])
    for d, m, Eb in dirichlet_faces(p):
        if p.limiter_jacobian in ("E", "exact"):
            W, dWi, _ = face_coefficient_derivatives(p, E, Eb, kap, kap, a, 0.5 * p.dx)
            di = W + dWi * (E - Eb)
        else:
            di = face_coefficient(p, E, Eb, kap, kap, a, 0.5 * p.dx)
        diag += np.where(m, dth * di, 0.0)
    return diag, rows, cols, vals


def full_jacobian(p, U, eh, dt, a, adot, T_fixed=None, nbt=None):
    """The whole scaled Newton matrix (unreduced), sparse, variable-major ordering:
    rows/cols [v * N + cell] for v in (e_c, n_1.., E).  D is lagged (frozen at U), keeps
    dD/dE ("E"), or keeps dD/dE and the opacity's species dependence ("exact"), which adds
    E-row entries in the species columns of the cell and of its neighbours."""
    ns, nm, N = p.ns, p.ns + 1, p.N
    M, Ucol, Lrow, Dloc, lt = local_blocks(p, U, eh, dt, a, adot, T_fixed)
    nbt = neighbor_table(p) if nbt is None else nbt
    ddiag, drows, dcols, dvals = diffusion_block(p, U[1 + ns], lt["kappa"], a, dt * p.theta, nbt)
    cells = np.arange(N)
    rows, cols, vals = [], [], []
    for r in range(nm):
        for s in range(nm):
            rows.append(r * N + cells); cols.append(s * N + cells); vals.append(M[:, r, s])
        rows.append(r * N + cells); cols.append(nm * N + cells); vals.append(Ucol[:, r])
        rows.append(nm * N + cells); cols.append(r * N + cells); vals.append(Lrow[:, r])
    rows.append(nm * N + cells); cols.append(nm * N + cells); vals.append(Dloc + ddiag)
    if p.limiter_jacobian == "exact":
        kdiag, krows, kcols, kvals = diffusion_kappa_block(p, U[1 + ns], lt["kappa"], a,
                                                           dt * p.theta, nbt)
        sk = p.grey["sk"]
        for X in range(ns):
            # d kappa / d n_X = sk_X / a^3; scaled entry d(f_E/u_E) / d(n_X/u_n)
            fac = sk[X] / a ** 3 * p.u_n / p.u_E
            rows.append(nm * N + cells); cols.append((1 + X) * N + cells); vals.append(fac * kdiag)
            for rr, cc, vv in zip(krows, kcols, kvals):
                rows.append(nm * N + rr); cols.append((1 + X) * N + cc); vals.append(fac * vv)
    for rr, cc, vv in zip(drows, dcols, dvals):
        rows.append(nm * N + rr); cols.append(nm * N + cc); vals.append(vv)
    J = sparse.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(p.nv * N, p.nv * N))
    return J.tocsr()
