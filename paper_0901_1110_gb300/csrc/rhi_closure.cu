// Host-side closure: the rate / cooling coefficient table and the grey spectral constants.
//
// The paper cites but does not print the rate and cooling formulas (Sec. 2.1, nLTE coupling);
// the closure is the project's: case-B recombination and its cooling in the forms of
// Hui & Gnedin (1997), collisional ionisation / excitation cooling, dielectronic recombination
// and bremsstrahlung in the forms of Cen (1992), as listed in the design notes.  As in Enzo the
// coefficients are tabulated over temperature and interpolated linearly inside the solve; the
// table nodes are T_i = 2^(i >> 6) (1 + (i & 63) / 64), i = 0 .. NBINS.
#include <cmath>
#include <limits>

#include "rhi_internal.cuh"

namespace rhi {

namespace {

constexpr double T_HI = 157807.0, T_HEI = 285335.0, T_HEII = 631515.0;

double hg97_caseB_rate(double T, double Tthr) {
    const double lam = 2.0 * Tthr / T;
    return 2.753e-14 * std::pow(lam, 1.5) / std::pow(1.0 + std::pow(lam / 2.740, 0.407), 2.242);
}
double hg97_caseB_cool(double T, double Tthr) {
    const double lam = 2.0 * Tthr / T;
    return 3.435e-30 * T * std::pow(lam, 1.970) / std::pow(1.0 + std::pow(lam / 2.250, 0.376), 3.720);
}
double hg97_HeII_caseB_rate(double T) { return 1.26e-14 * std::pow(2.0 * T_HEI / T, 0.75); }
double dielectronic(double T) {
    return 1.90e-3 * std::pow(T, -1.5) * std::exp(-470000.0 / T) * (1.0 + 0.3 * std::exp(-94000.0 / T));
}
double gaunt(double T) {
    const double d = 5.5 - std::log10(T);
    return 1.1 + 0.34 * std::exp(-d * d / 3.0);
}

void coefficients(double T, double* k) {
    const double sq = std::sqrt(T);
    const double d5 = 1.0 + std::sqrt(T / 1e5);
    const double brem = 1.42e-27 * gaunt(T) * sq;
    k[R_ALPHA_HII] = hg97_caseB_rate(T, T_HI);
    k[R_BETA_HI] = 5.85e-11 * sq * std::exp(-157809.1 / T) / d5;
    k[R_ALPHA_HEII] = hg97_HeII_caseB_rate(T) + dielectronic(T);
    k[R_BETA_HEI] = 2.38e-11 * sq * std::exp(-285335.4 / T) / d5;
    k[R_ALPHA_HEIII] = 2.0 * hg97_caseB_rate(T, T_HEII);
    k[R_BETA_HEII] = 5.68e-12 * sq * std::exp(-631515.0 / T) / d5;
    k[R_COOL_HI] = 7.50e-19 * std::exp(-118348.0 / T) / d5 +
                   1.27e-21 * sq * std::exp(-157809.1 / T) / d5;
    k[R_COOL_HII] = hg97_caseB_cool(T, T_HI) + brem;
    k[R_COOL_HEI] = 9.38e-22 * sq * std::exp(-285335.4 / T) / d5;
    k[R_COOL_HEII] = 4.95e-22 * sq * std::exp(-631515.0 / T) / d5 +
                     5.54e-17 * std::pow(T, -0.397) * std::exp(-473638.0 / T) / d5 +
                     K_BOLTZ * T * hg97_HeII_caseB_rate(T) +
                     1.24e-13 * std::pow(T, -1.5) * std::exp(-470000.0 / T) *
                         (1.0 + 0.3 * std::exp(-94000.0 / T)) +
                     brem;
    k[R_COOL_HEIII] = 8.0 * hg97_caseB_cool(T, T_HEII) + 4.0 * brem;
}

double node_T(int i) {
    return std::ldexp(1.0 + (double)(i & ((1 << TABLE_BITS) - 1)) / (double)(1 << TABLE_BITS),
                      i >> TABLE_BITS);
}

}  // namespace

std::vector<double2> build_rate_table() {
    std::vector<double> kv((size_t)(NBINS + 1) * NRATES);
    for (int i = 0; i <= NBINS; ++i) coefficients(node_T(i), &kv[(size_t)i * NRATES]);
    std::vector<double2> tab((size_t)NBINS * NRATES);
    for (int i = 0; i < NBINS; ++i) {
        const double w = node_T(i + 1) - node_T(i);
        for (int r = 0; r < NRATES; ++r) {
            const double k0 = kv[(size_t)i * NRATES + r], k1 = kv[(size_t)(i + 1) * NRATES + r];
            tab[(size_t)i * NRATES + r] = make_double2(k0, (k1 - k0) / w);
        }
    }
    return tab;
}

}  // namespace rhi

// ---------------------------------------------------------------------------------------------
// grey constants of eq. adaptive_spectrum by closed forms (Bose series, -ln(1 - e^-y), E_1)

namespace {

const double E_THR[3] = {13.6 * rhi::EV, 24.6 * rhi::EV, 54.4 * rhi::EV};
const double SIGMA_THR[3] = {6.30e-18, 7.42e-18, 1.575e-18};

// int_{y0}^inf y^n / (e^y - 1) dy, n = 2 or 3
double bose_moment(int n, double y0) {
    double s = 0.0;
    for (int k = 1; k < 4000; ++k) {
        const double e = std::exp(-k * y0);
        double t;
        if (n == 3)
            t = e * (y0 * y0 * y0 / k + 3.0 * y0 * y0 / ((double)k * k) + 6.0 * y0 / ((double)k * k * k) +
                     6.0 / ((double)k * k * k * k));
        else
            t = e * (y0 * y0 / k + 2.0 * y0 / ((double)k * k) + 2.0 / ((double)k * k * k));
        s += t;
        if (t < 1e-19 * s) break;
    }
    return s;
}

// int_{y0}^inf dy / (y (e^y - 1)) = sum_k E_1(k y0)
double bose_inverse(double y0) {
    double s = 0.0;
    for (int k = 1; k < 4000; ++k) {
        const double t = -std::expint(-(double)k * y0);
        s += t;
        if (t < 1e-19 * s) break;
    }
    return s;
}

}  // namespace

extern "C" int rhi_grey_constants(int spectrum, double param, int n_species, double* sk,
                                  double* pgam, double* ph, double* photon_energy) {
    if (!sk || !pgam || !ph || !photon_energy) return RHI_ERR_ARG;
    if (n_species != 0 && n_species != 1 && n_species != 3) return RHI_ERR_ARG;
    for (int X = 0; X < 3; ++X) sk[X] = pgam[X] = ph[X] = 0.0;
    if (spectrum == RHI_SPECTRUM_MONO) {
        const double hnu = param;
        if (!(hnu > 0.0)) return RHI_ERR_ARG;
        for (int X = 0; X < n_species; ++X) {
            if (hnu >= E_THR[X]) {
                const double r = hnu / E_THR[X];
                const double sig = SIGMA_THR[X] / (r * r * r);
                sk[X] = sig;
                pgam[X] = sig / hnu;
                ph[X] = sig * (1.0 - E_THR[X] / hnu);
            }
        }
        *photon_energy = hnu;
        return RHI_OK;
    }
    if (spectrum == RHI_SPECTRUM_BLACKBODY) {
        if (!(param > 0.0)) return RHI_ERR_ARG;
        const double kT = rhi::K_BOLTZ * param;
        const double y0 = E_THR[0] / kT;
        const double Z3 = bose_moment(3, y0), Z2 = bose_moment(2, y0);
        for (int X = 0; X < n_species; ++X) {
            const double yX = E_THR[X] / kT;
            const double pref = SIGMA_THR[X] * yX * yX * yX / Z3;
            const double I0 = -std::log1p(-std::exp(-yX));
            const double Im1 = bose_inverse(yX);
            sk[X] = pref * I0;
            pgam[X] = pref * Im1 / kT;
            ph[X] = pref * (I0 - yX * Im1);
        }
        *photon_energy = kT * Z3 / Z2;
        return RHI_OK;
    }
    if (spectrum == RHI_SPECTRUM_POWERLAW) {
        const double al = param;
        if (!(al < -1.0)) return RHI_ERR_ARG;
        const double E0 = E_THR[0];
        for (int X = 0; X < n_species; ++X) {
            const double tX = E_THR[X] / E0;
            sk[X] = SIGMA_THR[X] * std::pow(tX, al + 1.0) * (-al - 1.0) / (2.0 - al);
            pgam[X] = SIGMA_THR[X] * std::pow(tX, al) * (-al - 1.0) / ((3.0 - al) * E0);
            ph[X] = sk[X] - E_THR[X] * pgam[X];
        }
        *photon_energy = E0 * (-al) / (-al - 1.0);
        return RHI_OK;
    }
    return RHI_ERR_ARG;
}
