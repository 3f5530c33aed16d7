// Internal declarations shared by the CUDA translation units of librhi.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "rhi.h"
#include "rhi_fastdiv.h"

namespace rhi {

// ---------------------------------------------------------------------------------------------
// physical constants (CGS)
constexpr double C_LIGHT = 2.99792458e10;
constexpr double K_BOLTZ = 1.380649e-16;
constexpr double M_H = 1.67262192e-24;    // proton mass
constexpr double EV = 1.602176634e-12;
constexpr double GAMMA = 5.0 / 3.0;
constexpr double SIGMA_SB = 5.670374419e-5;   // erg cm^-2 s^-1 K^-4

// rate table: 2^TABLE_BITS bins per octave of T over [2^0, 2^TABLE_OCTAVES) K
constexpr int TABLE_BITS = 6;
constexpr int TABLE_OCTAVES = 30;
constexpr int NBINS = TABLE_OCTAVES << TABLE_BITS;
constexpr int NRATES = 11;
// largest double below 2^30
constexpr double T_TABLE_MAX = 1073741823.9999998807907104;

// rate columns
enum { R_ALPHA_HII = 0, R_BETA_HI, R_ALPHA_HEII, R_BETA_HEI, R_ALPHA_HEIII, R_BETA_HEII,
       R_COOL_HI, R_COOL_HII, R_COOL_HEI, R_COOL_HEII, R_COOL_HEIII };

// Host: node values and in-bin slopes of every coefficient, layout [bin][rate] of
// (value at the bin's lower node, slope); NBINS * NRATES entries.
std::vector<double2> build_rate_table();

// ---------------------------------------------------------------------------------------------
// per-step constants handed to kernels by value
struct StepParams {
    int nx, ny, nz;
    long long N;
    FastDiv fd_nx, fd_nxy;            // division by nx and nx * ny
    int per_x, per_y, per_z;          // periodic axes
    int dir_mask;                     // bit d: face d (x-, x+, y-, y+, z-, z+) is Dirichlet
    double Eb[6];                     // E on the Dirichlet faces
    double dx;
    double a, ia3, adot_a;            // a, 1/a^3, adot / a
    double dt, dth, dtm1;             // dt, dt theta, dt (theta - 1)
    double inv_a2dx2;                 // 1 / (a dx)^2
    double inv_adx;                   // 1 / (a dx)
    double half_adx;                  // a dx / 2
    double R_min;                     // limiter floor 1 / (a L)
    double kappa_floor;
    double m_grey;
    int isothermal, limiter;
    int limiter_newton;               // 1: keep dD/dE in the Newton matrix (non-symmetric S)
    double y_he;
    double u_e, u_n, u_E, iu_e, iu_n, iu_E;
    // dt theta times ratios of scalings for the scaled local blocks: M[0][s>0] (u_n / u_e),
    // M[r>0][0] (u_e / u_n), U column (u_E / u_e, u_E / u_n), L row (u_e / u_E, u_n / u_E)
    double sc_ne, sc_en, sc_Ee, sc_En, sc_eE, sc_nE;
    double sk[3], pg[3], ph[3];
    double tau;
    // LTE coupling (eq. LTE_coupling; no species): constant opacities, T = lte_cT e
    int lte;
    double kappa_total, kappa_planck, lte_cT;
    const double2* __restrict__ table;
};

// ---------------------------------------------------------------------------------------------
// grid helpers

struct Nbr {
    long long lo[3], hi[3];           // neighbour indices (valid only where the face exists)
    bool has_lo[3], has_hi[3];        // face carries flux
};

__device__ __forceinline__ void cell_coords(const StepParams& P, long long c, int& i, int& j,
                                            int& k) {
    const unsigned cu = (unsigned)c;
    const unsigned kk = fdiv(cu, P.fd_nxy);
    const unsigned r = cu - kk * P.fd_nxy.d;
    const unsigned jj = fdiv(r, P.fd_nx);
    k = (int)kk;
    j = (int)jj;
    i = (int)(r - jj * P.fd_nx.d);
}

__device__ __forceinline__ Nbr neighbours(const StepParams& P, long long c, int i, int j, int k) {
    Nbr b;
    const long long sx = 1, sy = P.nx, sz = (long long)P.nx * P.ny;
    const int n[3] = {P.nx, P.ny, P.nz};
    const int q[3] = {i, j, k};
    const long long s[3] = {sx, sy, sz};
    const int per[3] = {P.per_x, P.per_y, P.per_z};
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        if (q[ax] > 0) { b.lo[ax] = c - s[ax]; b.has_lo[ax] = true; }
        else if (per[ax]) { b.lo[ax] = c + (long long)(n[ax] - 1) * s[ax]; b.has_lo[ax] = true; }
        else { b.lo[ax] = c; b.has_lo[ax] = false; }
        if (q[ax] < n[ax] - 1) { b.hi[ax] = c + s[ax]; b.has_hi[ax] = true; }
        else if (per[ax]) { b.hi[ax] = c - (long long)(n[ax] - 1) * s[ax]; b.has_hi[ax] = true; }
        else { b.hi[ax] = c; b.has_hi[ax] = false; }
    }
    return b;
}

// ---------------------------------------------------------------------------------------------
// deterministic block reduction of a double; result valid in thread 0
template <int BLOCK>
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double warp_part[BLOCK / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) warp_part[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < BLOCK / 32; ++q) s += warp_part[q];
    }
    __syncthreads();
    return s;
}

// ---------------------------------------------------------------------------------------------
// kernel launch wrappers (defined in the .cu files); all return cudaGetLastError()

struct PhysBuffers {
    // state U^n
    const double* E_n;
    const double* n_n;      // ns * N
    const double* eh;       // e^n (specific energy before the step)
    const double* nH;
    const double* src;
    const double* Tiso;
    // iterate U (e_c, n, E) and its opacity
    const double* ec;       // may be null: e_c = 0
    const double* n;
    const double* E;
    const double* kap;
    const double* W;        // 3 * N lower-face coefficients (per unit time)
    const double* PQ;       // 6 * N Newton-matrix face entries (P then Q) or null
    double* g;              // (ns + 2) * N
    // outputs of the cell kernel
    double* diag;           // Schur diagonal with D lagged (scaled; the preconditioner's)
    double* diag_ns;        // Schur diagonal with dD/dE kept (when PQ is given)
    double* rhs;            // Schur right-hand side (scaled)
    double* fMt;            // (ns + 1) * N   M^-1 f_M (scaled)
    double* MiU;            // (ns + 1) * N   M^-1 U  (scaled)
    double* f_out;          // optional (ns + 2) * N scaled residual
    double* partials;       // per-block sums of the squared scaled residual
    double* U0;             // optional predictor output (ns + 2) * N
};

enum CellMode { MODE_PREP = 0, MODE_ITER = 1, MODE_PREP_PREDICT = 2, MODE_RESID = 3 };

cudaError_t launch_kappa(const StepParams& P, int ns, const double* n, double* kap,
                         cudaStream_t st);
cudaError_t launch_faces(const StepParams& P, const double* E, const double* kap, double* W,
                         double* PQ, double* K, cudaStream_t st);
// the face coefficients W alone, with the arithmetic of launch_faces for Newton matrix jm
// (limiter_jacobian), so that W is the same to the bit
cudaError_t launch_faces_w(const StepParams& P, int jm, const double* E, const double* kap,
                           double* W, cudaStream_t st);
cudaError_t launch_schur_kappa(const StepParams& P, int ns, const double* K, const double* fMt,
                               const double* MiU, double* PQ, double* diag_ns, double* rhs,
                               cudaStream_t st);
cudaError_t launch_export_faces(const StepParams& P, const double* W, const double* PQ,
                                double* S_lo, double* S_hi, cudaStream_t st);
cudaError_t launch_cell(const StepParams& P, int ns, int mode, const PhysBuffers& B,
                        int nblocks, cudaStream_t st);
int cell_block_size();
cudaError_t launch_update(const StepParams& P, int ns, double lam, const double* ec0,
                          const double* n0, const double* E0, const double* eh,
                          const double* nH, const double* sE, const double* fMt,
                          const double* MiU, double* ec1, double* n1, double* E1,
                          double* kap1, cudaStream_t st);
cudaError_t launch_finalize(const StepParams& P, int ns, const double* ec, double* eh,
                            cudaStream_t st);
cudaError_t launch_temperature(const StepParams& P, int ns, const double* e, const double* n,
                               const double* nH, double* T, cudaStream_t st);
cudaError_t launch_check_state(const StepParams& P, int ns, const double* E, const double* e,
                               const double* n, const double* nH, int* bad, cudaStream_t st);
cudaError_t launch_deposit(long long cell, double value, double* src, cudaStream_t st);
// block partials (nblocks of 256 threads) of the step's error estimate against the predictor
// Up: sum of q^pn, or max q when pn < 0
cudaError_t launch_time_error(const StepParams& P, int ns, const double* ec, const double* n,
                              const double* E, const double* Up, double pn, double* partials,
                              int nblocks, cudaStream_t st);

}  // namespace rhi
