/*
 * rhi.h -- C ABI of the GB300 implicit radiation / ionization / gas-energy step.
 *
 * One call of rhi_implicit_step advances the coupled system of Reynolds, Hayes, Paschos &
 * Norman (Sec. 3.1, eqs. RT-cons_energy, RT-chemical_ionization, RT-cons_radiation)
 *
 *     d e_c / dt = -2 (adot/a) e_c + G - Lambda
 *     d n_i / dt = alpha_ij n_e n_j - n_i Gamma_i
 *     d E   / dt = div(D grad E) - m (adot/a) E + 4 pi eta - c kappa E
 *
 * by one theta-scheme step (Sec. 3.2, eqs. energy/chemistry/radiation_simplified), solving the
 * nonlinear residual f(U) = 0 (eq. nonlinear_residual) with a globalised inexact Newton
 * iteration (Sec. 3.2), a cell-local Schur-complement elimination of the (e_c, n_i) blocks
 * (Sec. 3.2.1, eqs. newton_system2, schur_components, step_ia) and a multigrid-preconditioned
 * conjugate-gradient solve of the remaining 7-point system in E (Sec. 3.2.1, step (ii)).
 *
 * Conventions for every entry point:
 *  - Fields are cell-centred on an nx x ny x nz grid, flat index i + nx*(j + ny*k) (x fastest),
 *    FP64, CGS units, comoving (Sec. 2: n_i, E comoving; e specific energy in erg/g).
 *  - "n" arrays hold the independent species back to back: n_HI for n_species = 1, then
 *    n_HeI, n_HeII for n_species = 3 (n_species * N doubles).  n_HII, n_HeIII and n_e follow
 *    from element conservation (n_He = y_he * n_H).
 *  - Pointers flagged on_device = 1 are CUDA device pointers on the handle's device; 0 means
 *    host memory.  The library copies inputs and never keeps caller pointers; the caller owns
 *    all memory it passes.  Device work runs on the stream given to rhi_create; calls return
 *    after that work has completed.
 *  - Every function returns RHI_OK (0) or an RHI_ERR_* code; rhi_last_error(handle) gives a
 *    one-line reason.  On a failed rhi_implicit_step the state is left at U^n.
 */
#ifndef RHI_H
#define RHI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RHI_OK 0
#define RHI_ERR_ARG 1           /* invalid argument or size                                  */
#define RHI_ERR_CUDA 2          /* a CUDA call failed                                        */
#define RHI_ERR_NONCONVERGED 3  /* Newton did not reach newton_tol within max_newton         */
#define RHI_ERR_NONPHYSICAL 4   /* non-positive or non-finite state, or a CG breakdown       */
#define RHI_ERR_STATE 5         /* call order: no state set yet                              */

enum { RHI_BC_ZERO_FLUX = 0, RHI_BC_PERIODIC = 1, RHI_BC_DIRICHLET = 2 };
enum { RHI_GUESS_PREVIOUS = 0, RHI_GUESS_PREDICTOR = 1, RHI_GUESS_LEARNED = 2 };
/* physics model: non-LTE ionization chemistry (Sec. 2.1, n_species 1 or 3), or the LTE
   coupling of eq. LTE_coupling (n_species 0: gas and radiation energy only, constant total
   and Planck-mean opacities, T = (gamma - 1) mu m_H e / k_B) */
enum { RHI_MODEL_IONIZATION = 0, RHI_MODEL_LTE = 1 };
enum { RHI_PRECOND_JACOBI = 0, RHI_PRECOND_MG_FP64 = 1, RHI_PRECOND_MG_FP32 = 2 };
enum { RHI_SPECTRUM_MONO = 0, RHI_SPECTRUM_BLACKBODY = 1, RHI_SPECTRUM_POWERLAW = 2 };

/* Uniform Cartesian grid (Sec. 1: uniform grids only); dx = comoving cell width in cm. */
typedef struct {
    int nx, ny, nz;
    double dx;
} rhi_grid;

/* Boundary kind per face, order x-, x+, y-, y+, z-, z+; periodic faces come in pairs.
   A Dirichlet face holds the radiation energy density value[d] (erg cm^-3, > 0) on the face,
   half a cell from the centre of the cell next to it; the flux through it is
   D (E_b - E) / (a^2 dx dx/2) with the limiter's R over that distance and the cell's
   opacity.  The gas and species have no boundary fluxes (the path has no hydrodynamics). */
typedef struct {
    int kind[6];
    double value[6];
} rhi_bc;

/* Method and closure parameters.  Fill with rhi_params_default, then override. */
typedef struct {
    int n_species;          /* 1: H (HI); 3: H + He (HI, HeI, HeII); 0: the LTE model       */
    double y_he;            /* n_He / n_H; 0 when n_species = 1                              */
    double theta;           /* theta of the two-level scheme (Sec. 3.2)                      */
    int m_grey;             /* m of eq. cons_radiation (1 grey, 0 monochromatic)             */
    int isothermal;         /* 1: temperature held at its value at rhi_set_state; e_c = 0    */
    int limiter;            /* 1: eq. limiter; 0: D = c / (3 max(kappa, kappa_floor))         */
    double kappa_floor;     /* cm^-1, only without the limiter                               */
    double u_e, u_n, u_E;   /* scalings of eq. scalings: erg/g, cm^-3, erg/cm^3               */
    double tau;             /* fraction-to-boundary of the positivity cap (0 < tau < 1)      */
    double lam_min;         /* smallest line-search parameter                                */
    double mlp_gate;        /* learned guess: predicted changes below this keep U^n          */
    double mlp_ood;         /* learned guess: cells with a normalised feature |(x - mean) /
                               scale| above this keep U^n (0: no such gate)                 */
    int mlp_restart;        /* learned guess: Newton restarts from U^n when the learned start
                               has not converged after this many iterations, or stagnates
                               (||f|| above 0.9 of its value two iterations earlier); 0: never */
    int mlp_retry;          /* learned guess: after a step whose guess lost to U^n, this many
                               steps start from U^n without evaluating the network          */
    double growth_max;      /* watchdog line search: a full step may raise ||f|| up to
                               growth_max times the best ||f|| of the step ...               */
    int watchdog;           /* ... for at most this many Newton iterations in a row          */
    int limiter_jacobian;   /* 0: D lagged in the Newton matrix (symmetric S, CG);
                               1: dD/dE kept and only the opacity lagged, as Sec. 3.2.1
                               states (non-symmetric S, BiCGStab with the same V-cycle);
                               2: exact, dD/dE and D's opacity dependence on the species
                               kept (non-symmetric 7-point S, BiCGStab)                     */
    int max_newton;         /* Newton iterations per step                                    */
    int max_pcg;            /* CG iterations per Newton iteration                            */
    int guess;              /* RHI_GUESS_*                                                   */
    int precond;            /* RHI_PRECOND_*                                                 */
    int mg_levels;          /* multigrid levels including the finest                         */
    int mg_pre, mg_post;    /* weighted-Jacobi sweeps before / after the coarse correction   */
    int mg_coarse_sweeps;   /* weighted-Jacobi sweeps on the coarsest level                  */
    double mg_omega;        /* Jacobi weight                                                 */
    int vcycle_graph;       /* 1: the FP32 V-cycle is captured once as a CUDA graph and
                               replayed (on a library-owned stream ordered by events)       */
    int krylov_graph;       /* 1: each BiCGStab solve runs as one CUDA graph launch, its loop a
                               while node whose iterations decide on the device whether to
                               continue (no host round trip per iteration); 0: the same
                               kernels launched from the host, one read per iteration       */
    int mg_matrix;          /* the operator the multigrid hierarchy is built from: 1 (default)
                               the Newton matrix the Krylov method solves (with dD/dE kept a
                               non-symmetric 7-point matrix, whose coarse levels then carry
                               both couplings of each face); 0 the lagged-D matrix
                               (symmetric), as a preconditioner of the Newton matrix        */
    int predict_final;      /* 1: when the last two Newton residuals predict (quadratic
                               model, with a factor 10 of margin) that the full step ends the
                               iteration, its trial iterate is evaluated for f alone (no
                               Jacobian, no Schur system); if ||f|| is then not below the
                               tolerance, the iterate is evaluated again in full.  The
                               iterates and residuals are those of 0 (no prediction)         */
    double krylov_restart;  /* BiCGStab restarts (shadow residual set to the current residual)
                               each time ||r|| has fallen below this fraction of its value at
                               the last start; 0: only on stagnation (||r|| not 10% below its
                               best for 20 iterations); at most 8 restarts per solve.
                               Negative (default): 0.01 with the FP32 multigrid, else 0      */
    int dt_norm;            /* adaptive time steps (Sec. 3.2.3): 0 off; p >= 1 the p-norm and
                               -1 the max norm of eq. time_error_estimator                  */
    double dt_tau_tol;      /* tau_tol of eq. time_step_selection                            */
    int model;              /* RHI_MODEL_* (rhi_params_default(0) selects the LTE model)     */
    double kappa_total;     /* LTE: total opacity, cm^-1 (absorption and the limiter)        */
    double kappa_planck;    /* LTE: Planck-mean opacity, cm^-1 (emission)                    */
    double mu;              /* LTE: mean particle mass in units of m_H                       */
    /* grey constants per absorber (HI, HeI, HeII) of eq. adaptive_spectrum:
       kappa = sum sk_X n_X / a^3, Gamma_X = c pgam_X E / a^3, G = c E sum ph_X n_X / (a^3 rho) */
    double sk[3], pgam[3], ph[3];
    double photon_energy;   /* mean photon energy (erg) used by rhi_set_sources              */
} rhi_params;

#define RHI_MAX_HISTORY 64

typedef struct {
    int status;             /* RHI_OK or the error of the last step                          */
    int newton_its;         /* Newton iterations of the last step                            */
    int pcg_its;            /* CG iterations summed over the step                            */
    int vcycles;            /* preconditioner applications summed over the step              */
    int backtracks;         /* line-search halvings                                          */
    int lam_min_steps;      /* line searches that ended at lam_min                           */
    int guess_used;         /* RHI_GUESS_* actually used (learned falls back to previous)    */
    int launches;           /* kernel launches of the last step                              */
    int guess_restarts;     /* 1 when Newton abandoned the learned start for U^n (mlp_restart) */
    int krylov_fallbacks;   /* Newton iterations whose BiCGStab broke down and that took the
                               lagged-D direction (CG) instead                              */
    int host_syncs;         /* blocking device-to-host reads the step made (residual norms,
                               Krylov results, the final wait)                               */
    int krylov_stalls;      /* BiCGStab solves ended because ||r|| had not fallen by 10% in 20
                               iterations (the Newton step then uses that inexact solution)  */
    int final_predicted;    /* predict_final: trial iterates evaluated for f alone ...       */
    int final_missed;       /* ... of which did not converge and were evaluated again        */
    double res_initial;     /* ||f(U_0)|| (eq. rmsnorm, scaled)                              */
    double res_final;       /* ||f(U^{n+1})||                                                */
    double res_guess_prev;  /* ||f(U^n)|| when a learned guess was tried, else 0             */
    double ms;              /* device time of the last step, ms                              */
    double eps_loc;         /* eq. time_error_estimator of the last step (dt_norm != 0)      */
    double dt_next;         /* eq. time_step_selection: tau_tol dt / eps_loc (dt_norm != 0)  */
    double res_history[RHI_MAX_HISTORY];  /* ||f|| after 0, 1, .. Newton iterations      */
} rhi_stats;

typedef struct rhi_ctx* rhi_handle;

/* Defaults: theta 0.51 (Sec. 3.2), grey m = 1, limiter on, D lagged in the Newton matrix
   (limiter_jacobian 0), tau 0.99, lam_min 1/16, growth_max 1e3, watchdog 3, max_newton 50,
   max_pcg 200, previous-step guess, FP64 multigrid with 6 levels, 2 + 2 sweeps, 16 coarse
   sweeps, omega 0.9, V-cycle graph on, BiCGStab graph on, multigrid of the Newton matrix
   (mg_matrix 1), predict_final 1, krylov_restart -1 (0.01 with the FP32 multigrid, else 0),
   learned-guess gates mlp_gate 1e-3, mlp_ood 6,
   mlp_restart 12, mlp_retry 4, fixed steps (dt_norm 0) with tau_tol 0.01, scalings 1,
   kappa_floor 1e-40, mu 0.6, and the grey constants of 13.6 eV monochromatic radiation with a
   6.3e-18 cm^2 HI cross section.  n_species must be 0 (LTE model), 1 or 3.  Host computation
   only. */
int rhi_params_default(rhi_params* p, int n_species);

/* Grey constants of eq. adaptive_spectrum (Sec. 3.2.5) for an assumed spectrum chi(nu):
   RHI_SPECTRUM_MONO (param = photon energy, erg), RHI_SPECTRUM_BLACKBODY (param = T_B, K),
   RHI_SPECTRUM_POWERLAW (chi ~ nu^param, param < -1).  Cross sections are
   sigma_X (nu / nu_X)^-3 above thresholds 13.6 / 24.6 / 54.4 eV with sigma_X = 6.30e-18,
   7.42e-18, 1.575e-18 cm^2; integrals run from 13.6 eV up (eq. grey_definition).  Writes
   sk, pgam, ph (3 each; absorbers beyond n_species are 0) and the mean photon energy.
   Host computation only. */
int rhi_grey_constants(int spectrum, double param, int n_species, double* sk, double* pgam,
                       double* ph, double* photon_energy);

/* Creates a solver for one grid on the current CUDA device.  stream is a cudaStream_t (NULL:
   the legacy default stream).  Allocates every device buffer the step needs.  Errors:
   RHI_ERR_ARG for non-positive sizes, unpaired periodic faces, n_species not 0, 1 or 3, or
   out-of-range parameters; RHI_ERR_CUDA when allocation fails. */
int rhi_create(const rhi_grid* grid, const rhi_bc* bc, const rhi_params* params,
               void* stream, rhi_handle* out);

/* Sets the state U^n: E (N), e (N, specific gas energy), n (n_species * N), the comoving
   hydrogen density n_H (N) and the emissivity 4 pi eta (N, erg cm^-3 s^-1; NULL = 0).
   Requires E > 0, e > 0, n_H > 0 and every species (independent and derived) >= 0
   (RHI_ERR_NONPHYSICAL otherwise).  Isothermal runs fix the temperature here.  The learned
   guess's retry count (mlp_retry) carries over, so a host that hands its state back every
   step runs the same steps as one that leaves it on the device. */
int rhi_set_state(rhi_handle h, const double* E, const double* e, const double* n,
                  const double* n_H, const double* src, int on_device);

/* Adds point sources to the emissivity: source s puts photons_per_s[s] * photon_energy into
   the comoving volume dx^3 of cell (ijk[3s], ijk[3s+1], ijk[3s+2]).  Host arrays. */
int rhi_set_sources(rhi_handle h, int nsrc, const int* ijk, const double* photons_per_s);

/* One implicit step t^n -> t^n + dt at expansion factor a and adot = da/dt (both time
   levels use them).  newton_tol is epsilon of Sec. 3.2 (||f|| of eq. rmsnorm over scaled
   unknowns); lin_tol sets the inexact-Newton tolerance delta_k = lin_tol * ||f(U_k)||. */
int rhi_implicit_step(rhi_handle h, double dt, double a, double adot, double newton_tol,
                      double lin_tol);

/* Copies the current state out (E, e, n as in rhi_set_state). */
int rhi_get_state(rhi_handle h, double* E, double* e, double* n, int on_device);

/* Statistics of the last rhi_implicit_step. */
int rhi_get_stats(rhi_handle h, rhi_stats* out);

/* The first Newton linear system of a step from the current state with the previous-step
   guess (U_0 = U^n), without solving it: the scaled residual f (n_species + 2 blocks of N:
   e_c, n_1.., E; eq. nonlinear_residual divided by the scalings), the Schur matrix diagonal
   S_diag (N), its face entries S_lo (3 blocks of N: the entry coupling a cell to its -x, -y,
   -z neighbour) and S_hi (3 blocks of N: to its +x, +y, +z neighbour), given as positive
   numbers (the matrix entries are their negatives; 0 where a face carries no flux), and the
   Schur right-hand side rhs = L M^-1 f_M - f_E (N), all in scaled unknowns.  With
   limiter_jacobian = 1 the matrix is the non-symmetric one that keeps dD/dE.  Any output
   pointer may be NULL. */
int rhi_linearize(rhi_handle h, double dt, double a, double adot, double* f, double* S_diag,
                  double* S_lo, double* S_hi, double* rhs, int on_device);

/* Scaled residual f(U) of eq. nonlinear_residual (with eq. scalings) of the step from the
   current state over dt, at the given iterate U = (e_c, n_1 .. n_Ns, E), each N long
   (e_c = e - e^n).  Writes f ((N_s + 2) x N, may be NULL) and its RMS norm (eq. rmsnorm, may
   be NULL).  An inspection entry point: it uses the step's work buffers. */
int rhi_residual(rhi_handle h, double dt, double a, double adot, const double* U, double* f,
                 double* norm, int on_device);

/* Applies the configured preconditioner (one V-cycle or Jacobi) of the Schur matrix built by
   the last rhi_linearize to r (N), writing z (N). */
int rhi_precond_apply(rhi_handle h, const double* r, double* z, int on_device);

/* Per-kernel device time: with profiling on, every launch is bracketed by CUDA events on the
   handle's stream and accumulated per kernel name.  rhi_kernel_times writes up to max
   entries (names as NUL-terminated strings of at most 47 chars in names[48*i..], total ms,
   launch count) and returns the number of kernels (>= 0) or -RHI_ERR_*.
   rhi_set_profiling_names restricts the events to launches of the comma-separated kernel
   names (NULL or "" times every launch), so that timing one kernel leaves the others
   unbracketed. */
int rhi_set_profiling(rhi_handle h, int on);
int rhi_set_profiling_names(rhi_handle h, const char* names);
int rhi_kernel_times(rhi_handle h, int max, char* names, double* total_ms, int* launches);

/* Adaptive time stepping (Sec. 3.2.3; needs params.dt_norm != 0): implicit steps from the
   current state until t_end, the first of length dt0, each later one the dt_next of its
   predecessor, clamped to [dt_min, dt_max] and to the time left.  A step whose Newton
   iteration fails (no convergence, a non-physical iterate or a Krylov breakdown) is retried
   with half the step (the state is unchanged by a failed step), down to dt_min.  Writes the time reached and the number of steps taken; returns RHI_OK, or
   the error of a step that failed at dt_min, or RHI_ERR_NONCONVERGED after max_steps steps
   short of t_end. */
int rhi_advance(rhi_handle h, double t_end, double dt0, double dt_min, double dt_max, double a,
                double adot, double newton_tol, double lin_tol, int max_steps, double* t_reached,
                int* steps);

/* Learned Newton initial guess (an addition; Sec. 3.2 leaves the initial iterate free): a
   per-cell MLP 13 -> 64 -> 64 -> 64 -> 6 with SiLU predicting the state at t^{n+1} from the
   state at t^n and its change over the previous step.  Features: log10 E/u_E, log10 e/u_e,
   log10 of the HI, HeI, HeII fractions, log10 n_H/u_n, log10(dt Gamma_HI + 1e-30),
   log10(1 + 4 pi eta dt / E), log10(dt / 1e12 s), log10 E/E^{n-1}, log10 e/e^{n-1},
   logit x_HI - logit x_HI^{n-1}, log10(dt / dt^{n-1}) (the last four 0 before the first
   step; the library keeps the state before its last accepted step, also across
   rhi_set_state).  Outputs: log10 E'/E, log10 e'/e, logit of x_HI', logits of the He
   fractions (softmax).  Weights (FP32, RHI_MLP_NWEIGHTS): W1 (64x13, row major), b1 (64), W2
   (64x64), b2, W3 (64x64), b3, W4 (6x64), b4 (6), then the input normalisation mean (13) and
   scale (13).  Inference uses BF16 copies on the tensor cores with FP32 accumulation; training
   updates the FP32 weights with Adam using FP32 forward / backward kernels.  With guess =
   RHI_GUESS_LEARNED a step evaluates ||f|| at U^n and at the network's guess (cells whose
   predicted changes are all below params.mlp_gate keep U^n) and starts Newton from the
   smaller; rhi_stats.guess_used says which. */
#define RHI_MLP_IN 13
#define RHI_MLP_HID 64
#define RHI_MLP_OUT 6
#define RHI_MLP_NWEIGHTS (64 * 13 + 64 + 64 * 64 + 64 + 64 * 64 + 64 + 6 * 64 + 6 + 13 + 13)
int rhi_mlp_set_weights(rhi_handle h, const float* w, size_t n);
int rhi_mlp_get_weights(rhi_handle h, float* w, size_t n);
/* Features (N x 13, FP32) of the current state for a step of length dt at expansion a. */
int rhi_mlp_features(rhi_handle h, double dt, double a, float* X, int on_device);
/* Training targets (N x 6, FP32) of the step from the given earlier state (E, e, n as in
   rhi_set_state) to the current state. */
int rhi_mlp_targets(rhi_handle h, const double* E_old, const double* e_old,
                    const double* n_old, float* Y, int on_device);
/* The learned guess U_0 = (e_c, n_1 .. n_Ns, E) ((N_s + 2) x N) that rhi_implicit_step with
   RHI_GUESS_LEARNED would start from (before its comparison with U^n): the network's outputs
   decoded (E' = E 10^o0, e' = e 10^o1, x_HI' = 1 / (1 + exp(-o2)), He fractions by softmax of
   o3..o5), cells whose predicted changes all stay below params.mlp_gate keeping U^n. */
int rhi_mlp_guess(rhi_handle h, double dt, double a, double* U0, int on_device);
/* Network outputs Y (n x 6) for features X (n x 13) on the tensor cores (BF16 weights). */
int rhi_mlp_forward(rhi_handle h, const float* X, float* Y, long long n, int on_device);
/* Mean squared error over the n samples and its gradient wrt the FP32 weights (FP32
   forward / backward; the normalisation entries get 0). */
int rhi_mlp_loss_grad(rhi_handle h, const float* X, const float* Y, long long n, float* grad,
                      double* loss, int on_device);
/* Adam (beta 0.9 / 0.999) over the n samples in minibatches of `batch`, `epochs` passes, in
   sample order; writes the mean loss of the last epoch.  X and Y are device pointers. */
int rhi_mlp_train(rhi_handle h, const float* X, const float* Y, long long n, int epochs,
                  int batch, double lr, double* loss);

/* Allocation-free RMS norm (no counterpart in the paper; an addition for callers that may
   not allocate device memory, such as code running while a stream is captured into a CUDA
   graph, where cudaMalloc is not allowed, or an application that owns all device memory
   through its own pool).  Computes out[0] = sqrt(sum_{i<n} v[i]^2 / count), the norm of
   eq. rmsnorm when v holds the scaled residual and count = N (N_s + 2).
   v (n doubles) and out (1 double) are device pointers owned by the caller; stream is a
   cudaStream_t (NULL: legacy default stream); the call only enqueues work and returns.
   Scratch: a static device array of RHI_NOALLOC_MAX_COUNT / 256 doubles (1 MiB) that every
   GPU loading the library holds until the process exits; nothing is allocated.  n above
   RHI_NOALLOC_MAX_COUNT is rejected with RHI_ERR_ARG before any launch.  The first call on a
   device looks up the scratch address for that device (make it before any stream capture).
   Every call overwrites the whole scratch it uses and nothing in it needs to start at zero,
   but calls that overlap on the GPU (different streams or host threads) race on it.  The call
   clears a launch error still pending from earlier work of the calling host thread
   (cudaGetLastError) before it launches, and reports RHI_ERR_CUDA only for its own launches. */
#define RHI_NOALLOC_MAX_COUNT 33554432LL
int rhi_rms_norm_noalloc(const double* v, long long n, long long count, double* out,
                         void* stream);

const char* rhi_last_error(rhi_handle h);
const char* rhi_status_string(int status);
void rhi_destroy(rhi_handle h);

#ifdef __cplusplus
}
#endif

#endif /* RHI_H */
