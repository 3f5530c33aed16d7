// Cell-local physics of the implicit step: opacity, limiter face coefficients, the fused
// residual / Jacobian / Schur-elimination kernel, the Newton update with positivity cap, and
// small state kernels.  All FP64.
//
// Reference passages: Sec. 3.2 (theta scheme, eqs. energy/chemistry/radiation_simplified,
// operators mDE, mLe, mLn, mLE, residual eq. nonlinear_residual, RMS norm eq. rmsnorm),
// Sec. 3.2.1 (Newton matrix eqs. jacobian_matrix / jacobian_submatrices, Schur steps (i)-(iii),
// eqs. newton_system2, schur_components, step_ia), Sec. 3.2.2 (scalings eq. scalings),
// Sec. 2.2 (limiter eq. limiter).
#include "rhi_internal.cuh"

namespace rhi {

constexpr int CELL_BLOCK = 128;
int cell_block_size() { return CELL_BLOCK; }

// ---------------------------------------------------------------------------------------------
// opacity kappa = sum_X sk_X n_X / a^3

__global__ void k_kappa(const StepParams P, int ns, const double* __restrict__ n,
                        double* __restrict__ kap) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= P.N) return;
    if (ns == 0) { kap[c] = P.kappa_total; return; }          // LTE: constant opacity
    double s = P.sk[0] * n[c];
    if (ns == 3) s += P.sk[1] * n[P.N + c] + P.sk[2] * n[2 * P.N + c];
    kap[c] = P.ia3 * s;
}

cudaError_t launch_kappa(const StepParams& P, int ns, const double* n, double* kap,
                         cudaStream_t st) {
    const int b = 256;
    k_kappa<<<(unsigned)((P.N + b - 1) / b), b, 0, st>>>(P, ns, n, kap);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// face coefficients D / (a dx)^2 of each cell's three lower faces (eq. limiter)
//
// R = |E_b - E_a| / (a dx Ebar) floored at R_min; with q = max(|dE|, R_min a dx Ebar) and
// s = a dx Ebar, D = c s (2 kappa s + q) / (6 kappa^2 s^2 + 3 kappa q s + q^2): one division.
//
// With dD/dE kept in the Newton matrix (Sec. 3.2.1 lags only the opacity), the face between
// lower cell a and upper cell b (dE = E_b - E_a) contributes dt theta P to b's diagonal and
// -dt theta Q to (b, a), dt theta Q to a's diagonal and -dt theta P to (a, b), where
// P = W + (dW/dE_b) dE and Q = W - (dW/dE_a) dE.  With R dD/dR = -c q^2 (4 kappa s + q) s / den^2
// and t = dE / (E_a + E_b): P = W + R dD/dR (1 - t) / (a dx)^2, Q = W + R dD/dR (1 + t) / (a dx)^2
// (both = W where R sits at its floor).

//
// The exact Newton matrix also keeps D's opacity dependence: K = (1/2) (dW/dkappa) dE per face,
// with dD/dkappa = -c s^2 (12 kappa^2 s^2 + 12 kappa s q + q^2) / den^2 (the quotient rule on
// eq. limiter; each cell's kappa enters the face mean with weight 1/2).

struct FaceCoef { double W, P, Q, K; };

// JM: 0 W only; 1 W, P, Q (dD/dE kept); 2 W, P, Q, K (exact)
// The limiter's face coefficients depend on (s, dE) = (a dx Ebar, E_b - E_a) only through
// their ratio: W, P and Q, and K apart from its factor dE, are homogeneous of degree 0.  Their
// squares and the 1 / den^2 of the derivatives leave the FP64 range once Ebar falls below about
// 1e-90 (deep neutral gas after many absorbing steps), and the result turns into 0 / 0 or
// x * inf.  A faint face is therefore brought to s in [1, 2) by a power of two, which is exact;
// the test runs on the bit pattern (integer pipe), s > 0 and below 2^-64.
__device__ __forceinline__ void faint_rescale(double& s, double& dE) {
    const long long sb = __double_as_longlong(s);
    if (sb > 0 && sb < 0x3BF0000000000000LL) {
        const int e = ilogb(s);
        s = scalbn(s, -e);
        dE = scalbn(dE, -e);
    }
}

template <int JM, bool WONLY = false>
__device__ __forceinline__ FaceCoef face_coef(const StepParams& P, double Ea, double Eb,
                                              double ka, double kb) {
    constexpr bool PQ = JM >= 1;
    const double kap = 0.5 * (ka + kb);
    FaceCoef r;
    r.K = 0.0;
    if (P.limiter) {
        const double Esum = Ea + Eb;
        double s = Esum * P.half_adx;                           // a dx Ebar
        const double dE = Eb - Ea;
        double dEs = dE;                                        // dE on the scale of s
        faint_rescale(s, dEs);
        const double qraw = fabs(dEs);
        const double q = fmax(qraw, P.R_min * s);
        const double ks = kap * s;
        const double num = C_LIGHT * s * (2.0 * ks + q);
        const double den = 6.0 * ks * ks + 3.0 * ks * q + q * q;
        if (!PQ) {
            r.W = num / den * P.inv_a2dx2;
            r.P = r.Q = r.W;
            return r;
        }
        const double iden = 1.0 / den;
        r.W = num * iden * P.inv_a2dx2;
        if (WONLY) {
            r.P = r.Q = r.W;
            return r;
        }
        if (JM == 2)
            r.K = -0.5 * C_LIGHT * s * s * (12.0 * ks * ks + 12.0 * ks * q + q * q) * iden * iden *
                  P.inv_a2dx2 * dE;
        if (qraw > P.R_min * s) {
            // R dD/dR (1 -+ t) with t = dE / Esum; s / Esum = a dx / 2, so RdD t needs no division
            const double X = -C_LIGHT * q * q * (4.0 * ks + q) * iden * iden * P.inv_a2dx2;
            const double RdD = X * s;
            const double RdDt = X * dEs * P.half_adx;
            r.P = r.W + RdD - RdDt;
            r.Q = r.W + RdD + RdDt;
        } else {
            r.P = r.Q = r.W;
        }
        return r;
    }
    r.W = C_LIGHT / (3.0 * fmax(kap, P.kappa_floor)) * P.inv_a2dx2;
    r.P = r.Q = r.W;
    if (JM == 2 && kap > P.kappa_floor) r.K = -0.5 * r.W / kap * (Eb - Ea);
    return r;
}

// A Dirichlet face: the boundary value E_b sits on the face, half a cell from the centre, and
// the face's opacity is the cell's.  The coefficient is D / (a^2 dx dx/2) with R over that
// half-cell distance (s = a (dx/2) Ebar); Qd is the cell's Newton-diagonal entry
// W - dW/dE_c (E_b - E_c) and dWdk = dW/dkappa (exact matrix).
struct BoundaryFace { double W, Qd, dWdk; };

__device__ __forceinline__ BoundaryFace boundary_face(const StepParams& P, double E, double Eb,
                                                      double kap) {
    BoundaryFace r;
    if (P.limiter) {
        const double Esum = E + Eb;
        double s = 0.5 * Esum * P.half_adx;
        double dE = Eb - E;
        faint_rescale(s, dE);
        const double qraw = fabs(dE);
        const double q = fmax(qraw, P.R_min * s);
        const double ks = kap * s;
        const double den = 6.0 * ks * ks + 3.0 * ks * q + q * q;
        const double iden = 1.0 / den;
        r.W = 2.0 * C_LIGHT * s * (2.0 * ks + q) * iden * P.inv_a2dx2;
        r.Qd = r.W;
        if (P.limiter_newton >= 1 && qraw > P.R_min * s) {
            const double X = -2.0 * C_LIGHT * q * q * (4.0 * ks + q) * iden * iden * P.inv_a2dx2;
            r.Qd = r.W + X * s + X * dE * 0.5 * P.half_adx;
        }
        r.dWdk = -2.0 * C_LIGHT * s * s * (12.0 * ks * ks + 12.0 * ks * q + q * q) * iden * iden *
                 P.inv_a2dx2;
        return r;
    }
    r.W = 2.0 * C_LIGHT / (3.0 * fmax(kap, P.kappa_floor)) * P.inv_a2dx2;
    r.Qd = r.W;
    r.dWdk = kap > P.kappa_floor ? -r.W / kap : 0.0;
    return r;
}

// WONLY: the coefficients W alone (a trial iterate evaluated for its residual only), by the
// same arithmetic as the JM kernel's W
template <int JM, bool WONLY = false>
__global__ void __launch_bounds__(256) k_faces(const StepParams P, const double* __restrict__ E,
                                               const double* __restrict__ kap,
                                               double* __restrict__ W, double* __restrict__ PQv,
                                               double* __restrict__ Kv) {
    constexpr bool PQ = JM >= 1 && !WONLY;
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= P.N) return;
    int i, j, k;
    cell_coords(P, c, i, j, k);
    const Nbr b = neighbours(P, c, i, j, k);
    const double Ec = E[c], kc = kap[c];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        FaceCoef f{0.0, 0.0, 0.0, 0.0};
        if (b.has_lo[ax]) f = face_coef<JM, WONLY>(P, E[b.lo[ax]], Ec, kap[b.lo[ax]], kc);
        W[ax * P.N + c] = f.W;
        if (PQ) {
            PQv[ax * P.N + c] = f.P;
            PQv[(3 + ax) * P.N + c] = f.Q;
        }
        if (JM == 2 && !WONLY) Kv[ax * P.N + c] = f.K;
    }
}

cudaError_t launch_faces(const StepParams& P, const double* E, const double* kap, double* W,
                         double* PQ, double* K, cudaStream_t st) {
    const int b = 256;
    const unsigned g = (unsigned)((P.N + b - 1) / b);
    if (PQ && K) k_faces<2><<<g, b, 0, st>>>(P, E, kap, W, PQ, K);
    else if (PQ) k_faces<1><<<g, b, 0, st>>>(P, E, kap, W, PQ, nullptr);
    else k_faces<0><<<g, b, 0, st>>>(P, E, kap, W, nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_faces_w(const StepParams& P, int jm, const double* E, const double* kap,
                           double* W, cudaStream_t st) {
    const int b = 256;
    const unsigned g = (unsigned)((P.N + b - 1) / b);
    if (jm == 0) k_faces<0><<<g, b, 0, st>>>(P, E, kap, W, nullptr, nullptr);
    else if (jm == 1) k_faces<1, true><<<g, b, 0, st>>>(P, E, kap, W, nullptr, nullptr);
    else k_faces<2, true><<<g, b, 0, st>>>(P, E, kap, W, nullptr, nullptr);
    return cudaGetLastError();
}

// Exact Newton matrix: the E row of a cell couples to the species of the cell and of its
// face neighbours through D's opacity.  After the cell-local elimination
// dn_j = -M_j^-1 f_M,j - M_j^-1 U_j dE_j, face f (lower cell l, upper cell u, stored at u) adds,
// with rho_j = sum_X (dkappa/dn_X) (M^-1 U)_j,X and phi_j likewise with M^-1 f_M (scaled),
//   P_f -= K_f rho_u,  Q_f += K_f rho_l,
//   diag_u -= dt theta K_f rho_u,  diag_l += dt theta K_f rho_l,
//   rhs_u += dt theta K_f (phi_l + phi_u),  rhs_l -= dt theta K_f (phi_l + phi_u).
// Each thread owns its cell's three lower faces, so every write has one writer.
template <int NS>
__global__ void __launch_bounds__(256) k_schur_kappa(const StepParams P,
                                                     const double* __restrict__ K,
                                                     const double* __restrict__ fMt,
                                                     const double* __restrict__ MiU,
                                                     double* __restrict__ PQ,
                                                     double* __restrict__ diag_ns,
                                                     double* __restrict__ rhs) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long N = P.N;
    if (c >= N) return;
    int i, j, k;
    cell_coords(P, c, i, j, k);
    const Nbr b = neighbours(P, c, i, j, k);
    const double kfac = P.u_n * P.iu_E * P.ia3;     // d kappa / d n_X = sk_X / a^3, scaled
    auto rho = [&](long long q) {
        double s = 0.0;
#pragma unroll
        for (int X = 0; X < NS; ++X) s += P.sk[X] * MiU[(1 + X) * N + q];
        return kfac * s;
    };
    auto phi = [&](long long q) {
        double s = 0.0;
#pragma unroll
        for (int X = 0; X < NS; ++X) s += P.sk[X] * fMt[(1 + X) * N + q];
        return kfac * s;
    };
    const double rc = rho(c), pc = phi(c);
    double dd = 0.0, dr = 0.0;
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (b.has_lo[ax]) {
            const long long l = b.lo[ax];
            const double Kf = K[ax * N + c];
            PQ[ax * N + c] -= Kf * rc;
            PQ[(3 + ax) * N + c] += Kf * rho(l);
            dd -= Kf * rc;
            dr += Kf * (phi(l) + pc);
        }
        if (b.has_hi[ax]) {
            const long long h = b.hi[ax];
            const double Kh = K[ax * N + h];
            dd += Kh * rc;
            dr -= Kh * (pc + phi(h));
        }
    }
    diag_ns[c] += P.dth * dd;
    rhs[c] += P.dth * dr;
}

cudaError_t launch_schur_kappa(const StepParams& P, int ns, const double* K, const double* fMt,
                               const double* MiU, double* PQ, double* diag_ns, double* rhs,
                               cudaStream_t st) {
    const int b = 256;
    const unsigned g = (unsigned)((P.N + b - 1) / b);
    if (ns == 0) return cudaSuccess;                  // constant opacity: no coupling
    if (ns == 1) k_schur_kappa<1><<<g, b, 0, st>>>(P, K, fMt, MiU, PQ, diag_ns, rhs);
    else k_schur_kappa<3><<<g, b, 0, st>>>(P, K, fMt, MiU, PQ, diag_ns, rhs);
    return cudaGetLastError();
}

// Newton-matrix face entries of each cell for inspection: S_lo[ax] couples a cell to its
// lower neighbour, S_hi[ax] to its upper neighbour (positive numbers; the matrix entries are
// their negatives; 0 where the face carries no flux).
__global__ void k_export_faces(const StepParams P, const double* __restrict__ W,
                               const double* __restrict__ PQ, double* __restrict__ lo,
                               double* __restrict__ hi) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= P.N) return;
    int i, j, k;
    cell_coords(P, c, i, j, k);
    const Nbr b = neighbours(P, c, i, j, k);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        const double* Qa = PQ ? PQ + (3 + ax) * P.N : W + ax * P.N;
        const double* Pa = PQ ? PQ + ax * P.N : W + ax * P.N;
        lo[ax * P.N + c] = P.dth * Qa[c];
        hi[ax * P.N + c] = b.has_hi[ax] ? P.dth * Pa[b.hi[ax]] : 0.0;
    }
}

cudaError_t launch_export_faces(const StepParams& P, const double* W, const double* PQ,
                                double* S_lo, double* S_hi, cudaStream_t st) {
    const int b = 256;
    k_export_faces<<<(unsigned)((P.N + b - 1) / b), b, 0, st>>>(P, W, PQ, S_lo, S_hi);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// local reaction operators and their derivatives (eqs. mLe, mLn, mLE, jacobian_submatrices)

template <int NS>
struct Local {
    double L[NS + 1];          // L_e, L_n1 ..
    double LE;                 // local part of the E operator
    double dLx[NS + 1][NS + 1];
    double dLxE[NS + 1];
    double dLEx[NS + 1];
    double dLEE;
};

template <int NS, bool JAC>
__device__ __forceinline__ void local_model(const StepParams& P, double ec,
                                            const double (&n)[NS > 0 ? NS : 1],
                                            double E, double eh, double nH, double src,
                                            double Tfix, Local<NS>& o) {
    if constexpr (NS == 0) {
        // LTE coupling (eq. LTE_coupling): emission 4 pi eta = 4 kappa_P sigma T^4, heating
        // c kappa E / rho, cooling 4 pi eta / rho; T = lte_cT e
        const double rho = M_H * nH * (1.0 + 4.0 * P.y_he), irho = 1.0 / rho;
        const double e = eh + ec;
        const double T = P.isothermal ? Tfix : P.lte_cT * e;
        const double T2 = T * T;
        const double emis = 4.0 * P.kappa_planck * SIGMA_SB * T2 * T2;
        const double ckE = C_LIGHT * P.kappa_total * E;
        o.L[0] = P.isothermal ? 0.0 : (2.0 * P.adot_a * ec - ckE * irho + emis * irho);
        o.LE = P.m_grey * P.adot_a * E - src + ckE - emis;
        if constexpr (!JAC) return;
        const double demis = P.isothermal ? 0.0 : 16.0 * P.kappa_planck * SIGMA_SB * T2 * T * P.lte_cT;
        o.dLx[0][0] = P.isothermal ? 0.0 : 2.0 * P.adot_a + demis * irho;
        o.dLxE[0] = P.isothermal ? 0.0 : -C_LIGHT * P.kappa_total * irho;
        o.dLEx[0] = -demis;
        o.dLEE = P.m_grey * P.adot_a + C_LIGHT * P.kappa_total;
        return;
    } else {
    const double c = C_LIGHT, ia3 = P.ia3;
    const double nHe = P.y_he * nH;
    const double nHI = n[0];
    double nHeI = 0.0, nHeII = 0.0;
    if constexpr (NS == 3) { nHeI = n[1]; nHeII = n[2]; }
    const double nHII = nH - nHI;
    const double nHeIII = nHe - nHeI - nHeII;
    const double ne = nHII + nHeII + 2.0 * nHeIII;
    const double rho = M_H * (nH + 4.0 * nHe);
    const double irho = 1.0 / rho;
    const double e = eh + ec;
    const double ntot = nH + nHe + ne;
    double T, dT_dec, dT_dne;
    if (P.isothermal) {
        T = Tfix;
        dT_dec = 0.0;
        dT_dne = 0.0;
    } else {
        const double intot = 1.0 / ntot;
        dT_dec = (GAMMA - 1.0) * rho / K_BOLTZ * intot;     // T is proportional to e
        T = dT_dec * e;
        dT_dne = -T * intot;                                // d n_tot = d n_e
    }

    // tabulated coefficients: bin = binary exponent and top mantissa bits of clamped T
    const bool clamped = !(T >= 1.0 && T <= T_TABLE_MAX);
    const double Tc = fmin(fmax(T, 1.0), T_TABLE_MAX);
    const unsigned long long bits = (unsigned long long)__double_as_longlong(Tc);
    const int bin = (int)((bits >> (52 - TABLE_BITS)) - (1023ull << TABLE_BITS));
    const double Ti = __longlong_as_double((long long)(bits & ~((1ull << (52 - TABLE_BITS)) - 1ull)));
    const double dTi = Tc - Ti;
    const double2* row = P.table + (long long)bin * NRATES;
    double k[NRATES], dk[NRATES];
#pragma unroll
    for (int r = 0; r < NRATES; ++r) {
        const bool need = (NS == 3) || r == R_ALPHA_HII || r == R_BETA_HI || r == R_COOL_HI ||
                          r == R_COOL_HII;
        if (need) {
            const double2 v = __ldg(row + r);
            k[r] = fma(v.y, dTi, v.x);
            dk[r] = clamped ? 0.0 : v.y;
        } else {
            k[r] = 0.0;
            dk[r] = 0.0;
        }
    }
    const double C = k[R_COOL_HI] * nHI + k[R_COOL_HII] * nHII + k[R_COOL_HEI] * nHeI +
                     k[R_COOL_HEII] * nHeII + k[R_COOL_HEIII] * nHeIII;

    const double cE = c * E * ia3;
    const double GHI = P.pg[0] * cE, GHeI = P.pg[1] * cE, GHeII = P.pg[2] * cE;
    const double ne3 = ia3 * ne;
    const double B0 = k[R_BETA_HI] * nHI - k[R_ALPHA_HII] * nHII;
    o.L[1] = GHI * nHI + ne3 * B0;
    double B1 = 0.0, B2 = 0.0;
    if constexpr (NS == 3) {
        B1 = k[R_BETA_HEI] * nHeI - k[R_ALPHA_HEII] * nHeII;
        B2 = (k[R_BETA_HEII] + k[R_ALPHA_HEII]) * nHeII - k[R_BETA_HEI] * nHeI -
             k[R_ALPHA_HEIII] * nHeIII;
        o.L[2] = GHeI * nHeI + ne3 * B1;
        o.L[3] = GHeII * nHeII - GHeI * nHeI + ne3 * B2;
    }
    const double heat = P.ph[0] * nHI + P.ph[1] * nHeI + P.ph[2] * nHeII;
    const double G = cE * heat * irho;
    const double Lam = ne3 * C * irho;
    o.L[0] = P.isothermal ? 0.0 : (2.0 * P.adot_a * ec - G + Lam);
    const double kap = ia3 * (P.sk[0] * nHI + P.sk[1] * nHeI + P.sk[2] * nHeII);
    o.LE = P.m_grey * P.adot_a * E - src + c * kap * E;
    if constexpr (!JAC) return;

    const double dne[3] = {-1.0, -2.0, -1.0};
    const double dCdn[3] = {k[R_COOL_HI] - k[R_COOL_HII], k[R_COOL_HEI] - k[R_COOL_HEIII],
                            k[R_COOL_HEII] - k[R_COOL_HEIII]};
    const double dCdT = dk[R_COOL_HI] * nHI + dk[R_COOL_HII] * nHII + dk[R_COOL_HEI] * nHeI +
                        dk[R_COOL_HEII] * nHeII + dk[R_COOL_HEIII] * nHeIII;
    // energy row
    if (P.isothermal) {
#pragma unroll
        for (int s = 0; s <= NS; ++s) o.dLx[0][s] = 0.0;
        o.dLxE[0] = 0.0;
    } else {
        o.dLx[0][0] = 2.0 * P.adot_a + ne3 * dCdT * dT_dec * irho;
#pragma unroll
        for (int j = 0; j < NS; ++j)
            o.dLx[0][1 + j] = -cE * P.ph[j] * irho +
                              ia3 * irho * (dne[j] * C + ne * dCdn[j] + ne * dCdT * dT_dne * dne[j]);
        o.dLxE[0] = -c * ia3 * heat * irho;
    }
    // species rows: d/dx [A + ia3 n_e B] = dA/dx + ia3 (dn_e/dx B + n_e dB/dx|_T + n_e dB/dT dT/dx)
    const double dBdT0 = dk[R_BETA_HI] * nHI - dk[R_ALPHA_HII] * nHII;
    o.dLx[1][0] = ne3 * dBdT0 * dT_dec;
    o.dLx[1][1] = GHI + ia3 * (dne[0] * B0 + ne * (k[R_BETA_HI] + k[R_ALPHA_HII]) +
                               ne * dBdT0 * dT_dne * dne[0]);
    o.dLxE[1] = c * P.pg[0] * ia3 * nHI;
    if constexpr (NS == 3) {
        o.dLx[1][2] = ia3 * (dne[1] * B0 + ne * dBdT0 * dT_dne * dne[1]);
        o.dLx[1][3] = ia3 * (dne[2] * B0 + ne * dBdT0 * dT_dne * dne[2]);
        const double dBdT1 = dk[R_BETA_HEI] * nHeI - dk[R_ALPHA_HEII] * nHeII;
        o.dLx[2][0] = ne3 * dBdT1 * dT_dec;
        o.dLx[2][1] = ia3 * (dne[0] * B1 + ne * dBdT1 * dT_dne * dne[0]);
        o.dLx[2][2] = GHeI + ia3 * (dne[1] * B1 + ne * k[R_BETA_HEI] + ne * dBdT1 * dT_dne * dne[1]);
        o.dLx[2][3] = ia3 * (dne[2] * B1 - ne * k[R_ALPHA_HEII] + ne * dBdT1 * dT_dne * dne[2]);
        o.dLxE[2] = c * P.pg[1] * ia3 * nHeI;
        const double dBdT2 = (dk[R_BETA_HEII] + dk[R_ALPHA_HEII]) * nHeII - dk[R_BETA_HEI] * nHeI -
                             dk[R_ALPHA_HEIII] * nHeIII;
        o.dLx[3][0] = ne3 * dBdT2 * dT_dec;
        o.dLx[3][1] = ia3 * (dne[0] * B2 + ne * dBdT2 * dT_dne * dne[0]);
        o.dLx[3][2] = -GHeI + ia3 * (dne[1] * B2 + ne * (-k[R_BETA_HEI] + k[R_ALPHA_HEIII]) +
                                     ne * dBdT2 * dT_dne * dne[1]);
        o.dLx[3][3] = GHeII + ia3 * (dne[2] * B2 +
                                     ne * (k[R_BETA_HEII] + k[R_ALPHA_HEII] + k[R_ALPHA_HEIII]) +
                                     ne * dBdT2 * dT_dne * dne[2]);
        o.dLxE[3] = c * ia3 * (P.pg[2] * nHeII - P.pg[1] * nHeI);
    }
    o.dLEx[0] = 0.0;
#pragma unroll
    for (int j = 0; j < NS; ++j) o.dLEx[1 + j] = c * ia3 * P.sk[j] * E;
    o.dLEE = P.m_grey * P.adot_a + c * kap;
    }
}

// Gaussian elimination with partial pivoting for two right-hand sides (step (i), eq. step_ia)
template <int NM>
__device__ __forceinline__ void lu_solve2(double (&A)[NM][NM], double (&y)[NM], double (&z)[NM]) {
    double inv[NM];
#pragma unroll
    for (int k = 0; k < NM; ++k) {
        int p = k;
        double best = fabs(A[k][k]);
#pragma unroll
        for (int r = k + 1; r < NM; ++r) {
            const double v = fabs(A[r][k]);
            if (v > best) { best = v; p = r; }
        }
#pragma unroll
        for (int r = k + 1; r < NM; ++r) {
            if (r == p) {
#pragma unroll
                for (int c = k; c < NM; ++c) { const double t = A[k][c]; A[k][c] = A[r][c]; A[r][c] = t; }
                double t = y[k]; y[k] = y[r]; y[r] = t;
                t = z[k]; z[k] = z[r]; z[r] = t;
            }
        }
        inv[k] = 1.0 / A[k][k];
#pragma unroll
        for (int r = k + 1; r < NM; ++r) {
            const double m = A[r][k] * inv[k];
#pragma unroll
            for (int c = k + 1; c < NM; ++c) A[r][c] -= m * A[k][c];
            y[r] -= m * y[k];
            z[r] -= m * z[k];
        }
    }
#pragma unroll
    for (int k = NM - 1; k >= 0; --k) {
        double sy = y[k], sz = z[k];
#pragma unroll
        for (int c = k + 1; c < NM; ++c) { sy -= A[k][c] * y[c]; sz -= A[k][c] * z[c]; }
        y[k] = sy * inv[k];
        z[k] = sz * inv[k];
    }
}

// ---------------------------------------------------------------------------------------------
// fused residual / Jacobian / Schur kernel
//
// MODE_PREP:         U = (0, n^n, E^n); writes g^n = U^n + dt (theta - 1) L(U^n), f(U^n),
//                    and the Schur system at U^n.
// MODE_ITER:         U given; reads g; writes f(U) and the Schur system at U.
// MODE_PREP_PREDICT: writes g^n and the explicit predictor U^n - dt L(U^n) (capped).
// MODE_RESID:        U given; reads g; writes f(U) only (the same arithmetic as MODE_ITER).

template <int NS, int MODE>
__global__ void __launch_bounds__(CELL_BLOCK) k_cell(const StepParams P, const PhysBuffers B) {
    constexpr int NM = NS + 1, NV = NS + 2;
    const long long c = blockIdx.x * (long long)CELL_BLOCK + threadIdx.x;
    const long long N = P.N;
    double fsq = 0.0;
    if (c < N) {
        int i, j, k;
        cell_coords(P, c, i, j, k);
        const Nbr nb = neighbours(P, c, i, j, k);
        const bool prep = (MODE != MODE_ITER && MODE != MODE_RESID);
        constexpr bool JAC = MODE != MODE_PREP_PREDICT && MODE != MODE_RESID;
        const double* En = prep ? B.E_n : B.E;
        const double* nn = prep ? B.n_n : B.n;
        const double E = En[c];
        double n[NS > 0 ? NS : 1];
#pragma unroll
        for (int s = 0; s < NS; ++s) n[s] = nn[s * N + c];
        const double ec = (prep || B.ec == nullptr) ? 0.0 : B.ec[c];
        const double eh = B.eh[c], nH = B.nH[c], src = B.src[c];
        const double Tfix = P.isothermal ? B.Tiso[c] : 0.0;

        // diffusion: sum over faces W (E_c - E_nb); W sum for the lagged-D diagonal and, with
        // dD/dE kept, the Newton-matrix diagonal sum (P of own lower faces, Q of upper faces)
        double Dterm = 0.0, Wsum = 0.0, PQsum = 0.0;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const double wlo = B.W[ax * N + c];
            const double whi = nb.has_hi[ax] ? B.W[ax * N + nb.hi[ax]] : 0.0;
            Dterm += wlo * (E - En[nb.lo[ax]]) + whi * (E - En[nb.hi[ax]]);
            Wsum += wlo + whi;
            if (JAC && B.PQ) {
                PQsum += B.PQ[ax * N + c];
                if (nb.has_hi[ax]) PQsum += B.PQ[(3 + ax) * N + nb.hi[ax]];
            }
        }
        // Dirichlet faces of boundary cells (they carry no entry in the face arrays)
        double kb_term = 0.0;
        if (P.dir_mask) {
            const int q[3] = {i, j, k};
            const int ext[3] = {P.nx, P.ny, P.nz};
            // the cell's opacity at this iterate (the same sum as k_kappa)
            double kc;
            if constexpr (NS == 0) {
                kc = P.kappa_total;
            } else {
                double sk = P.sk[0] * n[0];
                if constexpr (NS == 3) sk += P.sk[1] * n[1] + P.sk[2] * n[2];
                kc = P.ia3 * sk;
            }
#pragma unroll
            for (int d = 0; d < 6; ++d) {
                const int ax = d >> 1;
                if ((P.dir_mask >> d & 1) && q[ax] == ((d & 1) ? ext[ax] - 1 : 0)) {
                    const double Eb = P.Eb[d];
                    const BoundaryFace bf = boundary_face(P, E, Eb, kc);
                    Dterm += bf.W * (E - Eb);
                    Wsum += bf.W;
                    PQsum += bf.Qd;
                    kb_term += bf.dWdk * (E - Eb);
                }
            }
        }

        Local<NS> lo;
        local_model<NS, JAC>(P, ec, n, E, eh, nH, src, Tfix, lo);
        if constexpr (NS > 0 && JAC) {
            // exact matrix: a Dirichlet face's opacity is the cell's, so its kappa derivative
            // joins the cell's own E-row species entries
            if (P.limiter_newton == 2 && kb_term != 0.0) {
#pragma unroll
                for (int X = 0; X < NS; ++X) lo.dLEx[1 + X] += kb_term * P.ia3 * P.sk[X];
            }
        }
        double Lf[NV];
#pragma unroll
        for (int v = 0; v <= NS; ++v) Lf[v] = lo.L[v];
        Lf[NV - 1] = Dterm + lo.LE;
        double U[NV];
        U[0] = ec;
#pragma unroll
        for (int s = 0; s < NS; ++s) U[1 + s] = n[s];
        U[NV - 1] = E;
        double g[NV];
        if (prep) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                g[v] = U[v] + P.dtm1 * Lf[v];
                B.g[v * N + c] = g[v];
            }
        } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) g[v] = B.g[v * N + c];
        }

        if (MODE == MODE_PREP_PREDICT || (MODE == MODE_PREP && B.U0)) {
            // explicit Euler predictor U^n - dt L(U^n) (eq. explicit_predictor), positivity cap;
            // MODE_PREP writes it when the step estimates its error against it (Sec. 3.2.3)
            double d[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) d[v] = -P.dt * Lf[v];
            double cap = 1.0;
            auto bound = [&](double q, double dq, double tiny) {
                if (dq < 0.0) cap = fmin(cap, fmax(P.tau * (q + tiny) / (-dq), 0.0));
            };
            bound(eh + ec, d[0], 0.0);
            bound(E, d[NV - 1], 0.0);
            if constexpr (NS >= 1) {
                bound(n[0], d[1], 1e-13 * nH);
                bound(nH - n[0], -d[1], 1e-13 * nH);
            }
            if constexpr (NS == 3) {
                const double nHe = P.y_he * nH;
                bound(n[1], d[2], 1e-13 * nHe);
                bound(n[2], d[3], 1e-13 * nHe);
                bound(nHe - n[1] - n[2], -d[2] - d[3], 1e-13 * nHe);
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) B.U0[v * N + c] = U[v] + cap * d[v];
        }
        if (MODE != MODE_PREP_PREDICT) {
            // scaled residual (eq. nonlinear_residual / eq. scalings)
            double fs[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const double f = U[v] + P.dth * Lf[v] - g[v];
                fs[v] = f * (v == NV - 1 ? P.iu_E : (v == 0 ? P.iu_e : P.iu_n));
                fsq += fs[v] * fs[v];
                if (B.f_out) B.f_out[v * N + c] = fs[v];
            }
            if constexpr (MODE != MODE_RESID) {
            // scaled local blocks (eq. schur_components); dt theta u_s / u_r products per step
            double M[NM][NM], y[NM], z[NM], Lr[NM];
#pragma unroll
            for (int r = 0; r < NM; ++r) {
#pragma unroll
                for (int s = 0; s < NM; ++s) {
                    const double sc = (r == 0) == (s == 0) ? P.dth : (r == 0 ? P.sc_ne : P.sc_en);
                    M[r][s] = (r == s ? 1.0 : 0.0) + lo.dLx[r][s] * sc;
                }
                z[r] = lo.dLxE[r] * (r == 0 ? P.sc_Ee : P.sc_En);
                Lr[r] = lo.dLEx[r] * (r == 0 ? P.sc_eE : P.sc_nE);
                y[r] = fs[r];
            }
            const double Dloc = 1.0 + P.dth * lo.dLEE;
            lu_solve2<NM>(M, y, z);                         // y = M^-1 f_M, z = M^-1 U
            double LMU = 0.0, LMf = 0.0;
#pragma unroll
            for (int r = 0; r < NM; ++r) { LMU += Lr[r] * z[r]; LMf += Lr[r] * y[r]; }
            B.diag[c] = Dloc - LMU + P.dth * Wsum;
            if (B.PQ) B.diag_ns[c] = Dloc - LMU + P.dth * PQsum;
            B.rhs[c] = LMf - fs[NV - 1];
#pragma unroll
            for (int r = 0; r < NM; ++r) {
                B.fMt[r * N + c] = y[r];
                B.MiU[r * N + c] = z[r];
            }
            }
        }
    }
    if (MODE != MODE_PREP_PREDICT) {
        const double s = block_sum<CELL_BLOCK>(fsq);
        if (threadIdx.x == 0) B.partials[blockIdx.x] = s;
    }
}

cudaError_t launch_cell(const StepParams& P, int ns, int mode, const PhysBuffers& B,
                        int nblocks, cudaStream_t st) {
    const dim3 g(nblocks), b(CELL_BLOCK);
    if (ns == 0) {
        if (mode == MODE_PREP) k_cell<0, MODE_PREP><<<g, b, 0, st>>>(P, B);
        else if (mode == MODE_ITER) k_cell<0, MODE_ITER><<<g, b, 0, st>>>(P, B);
        else if (mode == MODE_RESID) k_cell<0, MODE_RESID><<<g, b, 0, st>>>(P, B);
        else k_cell<0, MODE_PREP_PREDICT><<<g, b, 0, st>>>(P, B);
    } else if (ns == 1) {
        if (mode == MODE_PREP) k_cell<1, MODE_PREP><<<g, b, 0, st>>>(P, B);
        else if (mode == MODE_ITER) k_cell<1, MODE_ITER><<<g, b, 0, st>>>(P, B);
        else if (mode == MODE_RESID) k_cell<1, MODE_RESID><<<g, b, 0, st>>>(P, B);
        else k_cell<1, MODE_PREP_PREDICT><<<g, b, 0, st>>>(P, B);
    } else {
        if (mode == MODE_PREP) k_cell<3, MODE_PREP><<<g, b, 0, st>>>(P, B);
        else if (mode == MODE_ITER) k_cell<3, MODE_ITER><<<g, b, 0, st>>>(P, B);
        else if (mode == MODE_RESID) k_cell<3, MODE_RESID><<<g, b, 0, st>>>(P, B);
        else k_cell<3, MODE_PREP_PREDICT><<<g, b, 0, st>>>(P, B);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Newton update: step (iii) recovery, positivity cap, line-search fraction, new opacity.
// The cap keeps every bounded quantity q (e, E: bound 0; species: bound -1e-13 of the element
// total) above its bound by (1 - tau) of its current distance q + tiny.

template <int NS>
__global__ void __launch_bounds__(256) k_update(const StepParams P, double lam,
                                                const double* __restrict__ ec0,
                                                const double* __restrict__ n0,
                                                const double* __restrict__ E0,
                                                const double* __restrict__ eh,
                                                const double* __restrict__ nHa,
                                                const double* __restrict__ sE,
                                                const double* __restrict__ fMt,
                                                const double* __restrict__ MiU,
                                                double* __restrict__ ec1, double* __restrict__ n1,
                                                double* __restrict__ E1,
                                                double* __restrict__ kap1) {
    constexpr int NM = NS + 1;
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long N = P.N;
    if (c >= N) return;
    const double se = sE[c];
    double s[NM];
#pragma unroll
    for (int r = 0; r < NM; ++r) s[r] = (-fMt[r * N + c] - MiU[r * N + c] * se) * (r == 0 ? P.u_e : P.u_n);
    const double sEp = se * P.u_E;
    const double ec = ec0 ? ec0[c] : 0.0;
    double n[NS > 0 ? NS : 1];
#pragma unroll
    for (int j = 0; j < NS; ++j) n[j] = n0[j * N + c];
    const double E = E0[c], nH = nHa[c];
    // smallest fraction tau (q + tiny) / (-dq) over the decreasing quantities, kept as a
    // numerator / denominator pair (denominators > 0) so that one division remains.  The sign
    // test and the clamp at 0 read the bit pattern on the integer pipe (the FP64 pipe is this
    // kernel's bound): dq with its sign bit set is dq < 0 or -0, and -0 changes nothing (its
    // product below is 0); a value with its sign bit clear and below the +inf pattern is
    // +0, positive or +inf and kept, anything else (negative, NaN) clamps to 0, as fmax(v, 0)
    double cnum = 1.0, cden = 1.0;
    auto bound = [&](double q, double dq, double tiny) {
        if (__double_as_longlong(dq) < 0) {
            const double v = P.tau * (q + tiny);
            const long long vb = __double_as_longlong(v);
            const double num = (vb >= 0 && vb <= 0x7FF0000000000000LL) ? v : 0.0;
            if (num * cden < cnum * (-dq)) { cnum = num; cden = -dq; }
        }
    };
    bound(eh[c] + ec, s[0], 0.0);
    bound(E, sEp, 0.0);
    if constexpr (NS >= 1) {
        bound(n[0], s[1], 1e-13 * nH);
        bound(nH - n[0], -s[1], 1e-13 * nH);
    }
    if constexpr (NS == 3) {
        const double nHe = P.y_he * nH;
        bound(n[1], s[2], 1e-13 * nHe);
        bound(n[2], s[3], 1e-13 * nHe);
        bound(nHe - n[1] - n[2], -s[2] - s[3], 1e-13 * nHe);
    }
    const double cap = (cden == 1.0) ? cnum : cnum / cden;
    const double fr = fmin(lam, cap);
    ec1[c] = ec + fr * s[0];
    double ksum = 0.0;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
        const double v = n[j] + fr * s[1 + j];
        n1[j * N + c] = v;
        ksum += P.sk[j] * v;
    }
    E1[c] = E + fr * sEp;
    kap1[c] = NS == 0 ? P.kappa_total : P.ia3 * ksum;
}

cudaError_t launch_update(const StepParams& P, int ns, double lam, const double* ec0,
                          const double* n0, const double* E0, const double* eh,
                          const double* nH, const double* sE, const double* fMt,
                          const double* MiU, double* ec1, double* n1, double* E1,
                          double* kap1, cudaStream_t st) {
    const int b = 256;
    const unsigned g = (unsigned)((P.N + b - 1) / b);
    if (ns == 0)
        k_update<0><<<g, b, 0, st>>>(P, lam, ec0, n0, E0, eh, nH, sE, fMt, MiU, ec1, n1, E1, kap1);
    else if (ns == 1)
        k_update<1><<<g, b, 0, st>>>(P, lam, ec0, n0, E0, eh, nH, sE, fMt, MiU, ec1, n1, E1, kap1);
    else
        k_update<3><<<g, b, 0, st>>>(P, lam, ec0, n0, E0, eh, nH, sE, fMt, MiU, ec1, n1, E1, kap1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// small state kernels

__global__ void k_finalize(long long N, const double* __restrict__ ec, double* __restrict__ eh) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c < N) eh[c] += ec[c];           // e^{n+1} = e_h + e_c (Sec. 3.1)
}

cudaError_t launch_finalize(const StepParams& P, int, const double* ec, double* eh,
                            cudaStream_t st) {
    const int b = 256;
    k_finalize<<<(unsigned)((P.N + b - 1) / b), b, 0, st>>>(P.N, ec, eh);
    return cudaGetLastError();
}

__global__ void k_temperature(const StepParams P, int ns, const double* __restrict__ e,
                              const double* __restrict__ n, const double* __restrict__ nHa,
                              double* __restrict__ T) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= P.N) return;
    if (ns == 0) { T[c] = P.lte_cT * e[c]; return; }          // LTE
    const double nH = nHa[c], nHe = P.y_he * nH;
    const double nHI = n[c];
    const double nHeI = ns == 3 ? n[P.N + c] : 0.0, nHeII = ns == 3 ? n[2 * P.N + c] : 0.0;
    const double ne = (nH - nHI) + nHeII + 2.0 * (nHe - nHeI - nHeII);
    const double rho = M_H * (nH + 4.0 * nHe);
    T[c] = (GAMMA - 1.0) * rho * e[c] / (K_BOLTZ * (nH + nHe + ne));
}

cudaError_t launch_temperature(const StepParams& P, int ns, const double* e, const double* n,
                               const double* nH, double* T, cudaStream_t st) {
    const int b = 256;
    k_temperature<<<(unsigned)((P.N + b - 1) / b), b, 0, st>>>(P, ns, e, n, nH, T);
    return cudaGetLastError();
}

__global__ void k_check_state(const StepParams P, int ns, const double* __restrict__ E,
                              const double* __restrict__ e, const double* __restrict__ n,
                              const double* __restrict__ nHa, int* bad) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= P.N) return;
    const double nH = nHa[c], nHe = P.y_he * nH;
    const double nHI = ns >= 1 ? n[c] : 0.0;
    const double nHeI = ns == 3 ? n[P.N + c] : 0.0, nHeII = ns == 3 ? n[2 * P.N + c] : 0.0;
    const bool ok = (E[c] > 0.0) && (e[c] > 0.0) && (nH > 0.0) && (nHI >= 0.0) &&
                    (nH - nHI >= 0.0) && (nHeI >= 0.0) && (nHeII >= 0.0) &&
                    (nHe - nHeI - nHeII >= 0.0) && isfinite(E[c]) && isfinite(e[c]) &&
                    isfinite(nH);
    if (!ok) atomicOr(bad, 1);
}

cudaError_t launch_check_state(const StepParams& P, int ns, const double* E, const double* e,
                               const double* n, const double* nH, int* bad, cudaStream_t st) {
    const int b = 256;
    k_check_state<<<(unsigned)((P.N + b - 1) / b), b, 0, st>>>(P, ns, E, e, n, nH, bad);
    return cudaGetLastError();
}

__global__ void k_deposit(long long cell, double value, double* src) { src[cell] += value; }

cudaError_t launch_deposit(long long cell, double value, double* src, cudaStream_t st) {
    k_deposit<<<1, 1, 0, st>>>(cell, value, src);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Local error estimate of the step against the explicit predictor (eqs. typical_values,
// time_error_estimator): per scaled unknown q = |a - b| / (sqrt|a b| + 1); block partials of
// sum q^p, or of max q when p < 0 (the max norm)

template <int NS>
__global__ void __launch_bounds__(256) k_time_error(const StepParams P, const double* __restrict__ ec,
                                                    const double* __restrict__ n,
                                                    const double* __restrict__ E,
                                                    const double* __restrict__ Up, double pn,
                                                    double* __restrict__ partials) {
    constexpr int NV = NS + 2;
    const long long N = P.N;
    double acc = 0.0;
    for (long long c = blockIdx.x * 256LL + threadIdx.x; c < N; c += (long long)gridDim.x * 256) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const double iu = v == 0 ? P.iu_e : (v == NV - 1 ? P.iu_E : P.iu_n);
            const double a = (v == 0 ? (ec ? ec[c] : 0.0) : (v == NV - 1 ? E[c] : n[(v - 1) * N + c])) * iu;
            const double b = Up[v * N + c] * iu;
            const double q = fabs(a - b) / (sqrt(fabs(a * b)) + 1.0);
            if (pn < 0.0) acc = fmax(acc, q);
            else acc += (pn == 1.0) ? q : (pn == 2.0 ? q * q : pow(q, pn));
        }
    }
    // block reduction (sum or max) in a fixed order
    __shared__ double part[8];
    if (pn < 0.0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc = fmax(acc, __shfl_down_sync(0xffffffffu, acc, o));
    } else {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    }
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = part[0];
        for (int w = 1; w < 8; ++w) s = pn < 0.0 ? fmax(s, part[w]) : s + part[w];
        partials[blockIdx.x] = s;
    }
}

cudaError_t launch_time_error(const StepParams& P, int ns, const double* ec, const double* n,
                              const double* E, const double* Up, double pn, double* partials,
                              int nblocks, cudaStream_t st) {
    if (ns == 0) k_time_error<0><<<nblocks, 256, 0, st>>>(P, ec, n, E, Up, pn, partials);
    else if (ns == 1) k_time_error<1><<<nblocks, 256, 0, st>>>(P, ec, n, E, Up, pn, partials);
    else k_time_error<3><<<nblocks, 256, 0, st>>>(P, ec, n, E, Up, pn, partials);
    return cudaGetLastError();
}

}  // namespace rhi
