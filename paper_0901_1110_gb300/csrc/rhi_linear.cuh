// Declarations of the CG / multigrid kernels' launchers (rhi_linear.cu).
#pragma once

#include "rhi_internal.cuh"

namespace rhi {

// One level's 7-point operator, stored per face: the face below cell c along axis ax carries
// W[ax][c], the coupling of row c to its lower neighbour, and Wp[ax][c], the coupling of the
// lower neighbour's row to c:
//   (A x)_c = diag_c x_c - scale * sum_ax (W[ax]_c x_lo(ax) + Wp[ax]_hi(ax) x_hi(ax)).
// A symmetric operator has Wp = W (the same arrays); the Newton matrix that keeps dD/dE has
// Wp != W.  Both are 0 on zero-flux boundary faces.
template <typename T>
struct Op {
    int nx, ny, nz;
    long long N;
    FastDiv fd_nx, fd_nxy;
    int per[3];
    const T* diag;
    const T* W[3];       // per lower face: the coupling of the upper cell's row
    const T* Wp[3];      // per lower face: the coupling of the lower cell's row (= W: symmetric)
    T scale;
    const T* wid;        // omega / diag, read by the multigrid smoothers
    const T* loc;        // diag - scale * (sum of the row's six couplings); FP64 levels only
    const double* skip;  // when not null and *skip != 0 the kernel returns at once (the second
                         // half of a BiCGStab iteration after the solve converged at its middle)
};

// Non-symmetric 7-point operator (the Schur matrix with dD/dE kept):
// (A x)_c = diag_c x_c - scale * sum_ax (Q[ax]_c x_lo + P[ax]_hi x_hi), P and Q per lower face.
struct OpNS {
    int nx, ny, nz;
    long long N;
    FastDiv fd_nx, fd_nxy;
    int per[3];
    const double* diag;
    const double* P[3];
    const double* Q[3];
    double scale;
    const double* skip;  // as Op::skip
};

// largest level solved by one single-CTA launch (all coarse sweeps)
constexpr long long COARSE_MAX = 8192;

// device scalar slots of the Krylov iterations.  The BiCGStab loop keeps its control state
// on the device: S_THR (converged when r.r <= S_THR), S_MAXIT, the iteration count S_ITS, S_DONE
// (nothing left to do in this iteration), S_HALF (converged at the middle of an iteration:
// x += alpha M^-1 p only) and S_CONT (1 while another iteration follows).
// S_BEST / S_BESTIT: the smallest r.r so far and its iteration; S_STALL: the loop ended because
// r.r had not fallen below 0.81 of that best (10% in ||r||) for STALL_ITS iterations.
// Restarts: S_INNER (0: none) is a relative bound on r.r; once r.r falls below S_INNER times
// S_RR0, its value at the start or the last restart, or once the solve stagnates, the next
// iteration restarts from the current x and r with a fresh shadow vector rh = r (S_RST), at
// most MAX_RESTARTS times (S_NRST counts them).
enum { S_RZ = 0, S_PQ, S_ALPHA, S_BETA, S_RR, S_BREAK, S_TMP, S_RHO, S_OMEGA, S_SS, S_TS,
       S_TT, S_RV, S_DONE, S_ITS, S_THR, S_MAXIT, S_INNER, S_HALF, S_CONT, S_BEST, S_BESTIT,
       S_STALL, S_RR0, S_NRST, S_RST, S_NSCAL = 32 };
constexpr int STALL_ITS = 20;
constexpr int MAX_RESTARTS = 8;
enum { RED_SUM = 0, RED_ALPHA = 1, RED_BETA = 2, RED_BICG_ALPHA = 3, RED_BICG_OMEGA = 4,
       RED_BICG_RHO = 5, RED_MAX = 6, RED_BICG_START = 7, RED_BICG_SS = 8,
       RED_BICG_NEXT = 9 };

// number of blocks of the grid-stride streaming kernels (= number of partial sums)
int stream_blocks(long long N);

// timing / counting hook called around every launch
struct LaunchHook {
    virtual void begin(const char* name) = 0;
    virtual void end() = 0;
    virtual ~LaunchHook() {}
};

// Once per process, before the first multigrid launch: the shared-memory limit of the staged
// sweep and the address of its wait-timeout flag.
cudaError_t linear_kernels_init();
// The staged sweep's wait-timeout flag into *host (pinned), on stream st; and its reset.
cudaError_t bulk_wait_flag_read(int* host, cudaStream_t st);
cudaError_t bulk_wait_flag_clear(cudaStream_t st);

struct LinLaunch {
    cudaStream_t st;
    LaunchHook* hook;
    long long fine_N = -1;      // smoothing sweeps on a level of this size get their own name
    // device flag handed to the multigrid, conversion and BiCGStab second-half kernels: they
    // return at once while it is non-zero (null: always run)
    const double* skip = nullptr;
    LinLaunch(cudaStream_t s, LaunchHook* h);
    void begin(const char* name);
    cudaError_t end();

    cudaError_t matvec_dot(const Op<double>& A, const double* p, double* q, double* part,
                           int& nparts);
    cudaError_t cg_xr(long long N, const double* scal, double* x, double* r, const double* p,
                      const double* q, double* part, int& nparts);
    cudaError_t cg_p(long long N, const double* scal, const double* z, double* p, int first);
    cudaError_t jacobi_dot(long long N, const double* r, const double* diag, double* z,
                           double* part, int& nparts);
    cudaError_t dot(long long N, const double* a, const double* b, double* part, int& nparts);
    cudaError_t cg_init(long long N, const double* b, double* r, double* x, double* part,
                        int& nparts);
    cudaError_t reduce(const double* part, int n, double* scal, int op, int slot);
    // the reductions of the device-controlled BiCGStab loop (RED_BICG_START / _SS / _NEXT);
    // cond: the CUDA-graph conditional handle the loop's continue flag is written to (0: none)
    cudaError_t reduce_loop(const double* part, int n, double* scal, int op,
                            unsigned long long cond);
    // BiCGStab (right-preconditioned) building blocks
    cudaError_t matvec_ns(const OpNS& A, const double* x, double* y, const double* w1,
                          int two_dots, double* part, int& nparts);
    cudaError_t bicg_init(long long N, const double* b, double* r, double* rh, double* x,
                          double* part, int& nparts);
    // first: 1 p = r; 0 the update; -1 decided on the device (p = r, and rh = r when rh is
    // given, at S_ITS = 0 or after a restart)
    cudaError_t bicg_p(long long N, const double* scal, const double* r, const double* v,
                       double* p, int first, double* rh = nullptr);
    cudaError_t bicg_s(long long N, const double* scal, const double* r, const double* v,
                       double* s, double* part, int& nparts);
    cudaError_t bicg_xr(long long N, const double* scal, double* x, const double* ph,
                        const double* sh, const double* s, const double* t, double* r,
                        const double* rh, double* part, int& nparts);
    cudaError_t axpy(long long N, const double* scal, int slot, const double* p, double* x);
    // the x / r update of the device-controlled loop: converged at the middle of the
    // iteration (S_HALF) x += alpha ph only; after a breakdown nothing
    cudaError_t bicg_xr_loop(long long N, const double* scal, double* x, const double* ph,
                             const double* sh, const double* s, const double* t, double* r,
                             const double* rh, double* part, int& nparts);
    cudaError_t from_f32(long long N, const float* x, double* z);
    cudaError_t copy(long long N, const double* a, double* b);

    template <typename T>
    cudaError_t smooth(const Op<T>& A, const T* b, const T* xin, T* xout, T omega, int first);
    // every sweep of a level of at most COARSE_MAX cells in one single-CTA launch; the result
    // ends in x when sweeps is odd, else in xt
    template <typename T>
    cudaError_t coarse_solve(const Op<T>& A, const T* b, T* x, T* xt, T omega, int sweeps);
    template <typename T>
    cudaError_t restrict_res(const Op<T>& A, const T* b, const T* x, int cnx, int cny, int cnz,
                             T* bc);
    template <typename T>
    cudaError_t prolong(int nx, int ny, int nz, int cnx, int cny, const T* xc, T* xf);
    // coarse operator of A: diagonal dc (local part; diag_faces adds the couplings), W-type
    // face arrays wc[3] and, for a non-symmetric A, Wp-type face arrays wpc[3] (else null)
    template <typename TF, typename TC>
    cudaError_t coarsen(const Op<TF>& A, int cnx, int cny, int cnz, TC* dc, TC* const* wc,
                        TC* const* wpc);
    template <typename T>
    cudaError_t diag_faces(const Op<T>& A, T* diag);
    // per cell of a level: wid = omega / diag (smoothers) and, if loc is not null,
    // loc = diag - scale * (six faces) (FP64 restriction), evaluated in TF and rounded to TO
    template <typename TF, typename TO>
    cudaError_t level_prep(const Op<TF>& A, double omega, TO* wid, TO* loc);
    // FP32 copy of an FP64 operator with the scale folded into the faces (wp null: symmetric)
    cudaError_t cast_op(const Op<double>& A, float* d, float* const* w, float* const* wp);
    cudaError_t to_f32(long long N, const double* a, float* b);
    cudaError_t from_f32_dot(long long N, const float* x, const double* r, double* z,
                             double* part, int& nparts);
};

}  // namespace rhi
