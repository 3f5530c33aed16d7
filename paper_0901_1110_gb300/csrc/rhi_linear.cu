// Scalar Schur-system solve (Sec. 3.2.1, step (ii)): conjugate gradients on the 7-point
// matrix S, preconditioned by one geometric multigrid V-cycle (FP64, or FP32 for the mixed-
// precision form) or by Jacobi.  Reductions are deterministic: per-block partial sums are
// added in a fixed order by a single block.
//
// Operator of a level: (A x)_c = diag_c x_c - scale * sum_ax (W[ax]_c x_lo + Wp[ax]_hi x_hi),
// stored per lower face (0 on zero-flux boundary faces): W couples the upper cell's row to the
// lower cell, Wp the lower cell's row to the upper cell.  Symmetric levels pass Wp = W.
#include "rhi_linear.cuh"

#include <type_traits>

namespace rhi {

constexpr int LIN_BLOCK = 256;
constexpr int RED_BLOCK = 1024;

// the second half of a converged BiCGStab iteration returns at once
__device__ __forceinline__ bool skipped(const double* skip) { return skip && *skip != 0.0; }

int stream_blocks(long long N) {
    const long long want = (N + LIN_BLOCK - 1) / LIN_BLOCK;
    const long long cap = 152LL * 16;                 // 16 resident blocks per SM x 152 SMs
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

template <typename T>
__device__ __forceinline__ void coords3(const Op<T>& A, long long c, int& i, int& j, int& k) {
    const unsigned cu = (unsigned)c;
    const unsigned kk = fdiv(cu, A.fd_nxy);
    const unsigned r = cu - kk * A.fd_nxy.d;
    const unsigned jj = fdiv(r, A.fd_nx);
    k = (int)kk;
    j = (int)jj;
    i = (int)(r - jj * A.fd_nx.d);
}

// coordinates of index c on an nx x ny x nz grid given the dividers of nx and nx * ny
__device__ __forceinline__ void coords_fd(long long c, const FastDiv& fx, const FastDiv& fxy,
                                          int& i, int& j, int& k) {
    const unsigned cu = (unsigned)c;
    const unsigned kk = fdiv(cu, fxy);
    const unsigned r = cu - kk * fxy.d;
    const unsigned jj = fdiv(r, fx);
    k = (int)kk;
    j = (int)jj;
    i = (int)(r - jj * fx.d);
}

// sum over the six neighbours of c of W_face x_neighbour (the off-diagonal part of row c
// before the scale)
template <typename T, typename TX>
__device__ __forceinline__ T off_row(const Op<T>& A, const TX* __restrict__ x, long long c,
                                     int i, int j, int k) {
    const long long sx = 1, sy = A.nx, sz = (long long)A.nx * A.ny;
    const int n[3] = {A.nx, A.ny, A.nz};
    const int q[3] = {i, j, k};
    const long long s[3] = {sx, sy, sz};
    const int per[3] = {A.per[0], A.per[1], A.per[2]};
    T off = T(0);
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
        long long lo, hi;
        bool has_hi = true;
        if (q[ax] > 0) lo = c - s[ax];
        else lo = c + (long long)(n[ax] - 1) * s[ax];            // W = 0 there unless periodic
        if (q[ax] < n[ax] - 1) hi = c + s[ax];
        else if (per[ax]) hi = c - (long long)(n[ax] - 1) * s[ax];
        else { hi = c; has_hi = false; }
        const T wlo = A.W[ax][c];
        off += wlo * T(x[lo]);
        if (has_hi) off += A.Wp[ax][hi] * T(x[hi]);
    }
    return off;
}

// (A x)_c with the six neighbours of c
template <typename T, typename TX>
__device__ __forceinline__ T apply_row(const Op<T>& A, const TX* __restrict__ x, long long c,
                                       int i, int j, int k, T xc) {
    return A.diag[c] * xc - A.scale * off_row(A, x, c, i, j, k);
}

// one weighted-Jacobi update of cell c from the off-diagonal sum:
// x + omega (b - A x) / diag = (1 - omega) x + (omega / diag) (b + scale off)
template <typename T>
__device__ __forceinline__ T jacobi_update(T xc, T b, T wi, T scale, T off, T omega) {
    return (T(1) - omega) * xc + wi * (b + scale * off);
}

// ---------------------------------------------------------------------------------------------
// CG building blocks (FP64)

__global__ void __launch_bounds__(LIN_BLOCK) k_matvec_dot(const Op<double> A,
                                                          const double* __restrict__ p,
                                                          double* __restrict__ q,
                                                          double* __restrict__ partials) {
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < A.N;
         c += (long long)gridDim.x * LIN_BLOCK) {
        int i, j, k;
        coords3(A, c, i, j, k);
        const double pc = p[c];
        const double v = apply_row(A, p, c, i, j, k, pc);
        q[c] = v;
        acc += pc * v;
    }
    const double s = block_sum<LIN_BLOCK>(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// x += alpha p; r -= alpha q; partial r.r      (alpha = scal[S_ALPHA])
__global__ void __launch_bounds__(LIN_BLOCK) k_cg_xr(long long N, const double* __restrict__ scal,
                                                     double* __restrict__ x, double* __restrict__ r,
                                                     const double* __restrict__ p,
                                                     const double* __restrict__ q,
                                                     double* __restrict__ partials) {
    const double alpha = scal[S_ALPHA];
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < N;
         c += (long long)gridDim.x * LIN_BLOCK) {
        x[c] += alpha * p[c];
        const double rv = r[c] - alpha * q[c];
        r[c] = rv;
        acc += rv * rv;
    }
    const double s = block_sum<LIN_BLOCK>(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// p = z + beta p    (beta = scal[S_BETA]); first: p = z
__global__ void __launch_bounds__(LIN_BLOCK) k_cg_p(long long N, const double* __restrict__ scal,
                                                    const double* __restrict__ z,
                                                    double* __restrict__ p, int first) {
    const double beta = first ? 0.0 : scal[S_BETA];
    for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < N;
         c += (long long)gridDim.x * LIN_BLOCK)
        p[c] = first ? z[c] : z[c] + beta * p[c];
}

// z = r / diag; partial r.z
__global__ void __launch_bounds__(LIN_BLOCK) k_jacobi_dot(long long N, const double* __restrict__ r,
                                                          const double* __restrict__ diag,
                                                          double* __restrict__ z,
                                                          double* __restrict__ partials,
                                                          const double* skip) {
    if (skipped(skip)) return;
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < N;
         c += (long long)gridDim.x * LIN_BLOCK) {
        const double rv = r[c];
        const double zv = rv / diag[c];
        z[c] = zv;
        acc += rv * zv;
    }
    const double s = block_sum<LIN_BLOCK>(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// partial a.b
__global__ void __launch_bounds__(LIN_BLOCK) k_dot(long long N, const double* __restrict__ a,
                                                   const double* __restrict__ b,
                                                   double* __restrict__ partials) {
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < N;
         c += (long long)gridDim.x * LIN_BLOCK)
        acc += a[c] * b[c];
    const double s = block_sum<LIN_BLOCK>(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// r = b, x = 0; partial r.r
__global__ void __launch_bounds__(LIN_BLOCK) k_cg_init(long long N, const double* __restrict__ b,
                                                       double* __restrict__ r,
                                                       double* __restrict__ x,
                                                       double* __restrict__ partials) {
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < N;
         c += (long long)gridDim.x * LIN_BLOCK) {
        const double v = b[c];
        r[c] = v;
        x[c] = 0.0;
        acc += v * v;
    }
    const double s = block_sum<LIN_BLOCK>(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Sum of partials in a fixed order, then a scalar update:
//   SUM_TO(k):   scal[k] = sum
//   SUM_ALPHA:   scal[S_PQ] = sum; scal[S_ALPHA] = scal[S_RZ] / sum (breakdown flag if <= 0)
//   SUM_BETA:    scal[S_BETA] = sum / scal[S_RZ]; scal[S_RZ] = sum
__global__ void __launch_bounds__(RED_BLOCK) k_reduce(const double* __restrict__ partials, int n,
                                                      double* __restrict__ scal, int op,
                                                      int slot, const double* skip) {
    if (skipped(skip)) return;
    // the BiCGStab updates carry a second set of partials after the first n
    const bool two = op == RED_BICG_OMEGA || op == RED_BICG_RHO;
    if (op == RED_MAX) {                        // max of non-negative partials
        __shared__ double wmax[RED_BLOCK / 32];
        double m = 0.0;
        for (int q = threadIdx.x; q < n; q += RED_BLOCK) m = fmax(m, partials[q]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int q = 1; q < RED_BLOCK / 32; ++q) m = fmax(m, wmax[q]);
            scal[slot] = fmax(m, wmax[0]);
        }
        return;
    }
    double acc = 0.0, acc2 = 0.0;
    for (int q = threadIdx.x; q < n; q += RED_BLOCK) {
        acc += partials[q];
        if (two) acc2 += partials[n + q];
    }
    const double s = block_sum<RED_BLOCK>(acc);
    const double s2 = two ? block_sum<RED_BLOCK>(acc2) : 0.0;
    if (threadIdx.x == 0) {
        if (op == RED_SUM) {
            scal[slot] = s;
        } else if (op == RED_ALPHA) {
            scal[S_PQ] = s;
            if (!(s > 0.0)) scal[S_BREAK] = 1.0;
            scal[S_ALPHA] = (s > 0.0) ? scal[S_RZ] / s : 0.0;
        } else if (op == RED_BETA) {
            scal[S_BETA] = s / scal[S_RZ];
            scal[S_RZ] = s;
        } else if (op == RED_BICG_ALPHA) {          // s = rh.v
            scal[S_RST] = 0.0;                      // a restart's p and rh are in place
            scal[S_RV] = s;
            if (!(s != 0.0)) scal[S_BREAK] = 1.0;
            scal[S_ALPHA] = (s != 0.0) ? scal[S_RHO] / s : 0.0;
        } else if (op == RED_BICG_OMEGA) {          // partials: t.s then t.t
            const double tt = s2;
            scal[S_TS] = s;
            scal[S_TT] = tt;
            scal[S_OMEGA] = (tt > 0.0) ? s / tt : 0.0;
            if (!(tt > 0.0)) scal[S_BREAK] = 1.0;
        } else {                                    // RED_BICG_RHO: partials r.r then rh.r
            const double rho = s2;
            scal[S_RR] = s;
            scal[S_BETA] = (rho / scal[S_RHO]) * (scal[S_ALPHA] / scal[S_OMEGA]);
            scal[S_RHO] = rho;
            if (!(rho != 0.0)) scal[S_BREAK] = 1.0;
        }
    }
}

// ---------------------------------------------------------------------------------------------
// BiCGStab building blocks (FP64), right preconditioning

// y = A x with the non-symmetric operator; partials w1.y (and y.y when TWO)
template <bool TWO>
__global__ void __launch_bounds__(LIN_BLOCK) k_matvec_ns(const OpNS A, const double* __restrict__ x,
                                                         double* __restrict__ y,
                                                         const double* __restrict__ w1,
                                                         double* __restrict__ partials) {
    if (skipped(A.skip)) return;
    double d1 = 0.0, d2 = 0.0;
    const long long sz = (long long)A.nx * A.ny;
    for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < A.N;
         c += (long long)gridDim.x * LIN_BLOCK) {
        int i, j, k;
        coords_fd(c, A.fd_nx, A.fd_nxy, i, j, k);
        const int q[3] = {i, j, k};
        const int n[3] = {A.nx, A.ny, A.nz};
        const long long s[3] = {1, A.nx, sz};
        double off = 0.0;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const long long lo = q[ax] > 0 ? c - s[ax] : c + (long long)(n[ax] - 1) * s[ax];
            off += A.Q[ax][c] * x[lo];                // 0 on zero-flux boundary faces
            long long hi = -1;
            if (q[ax] < n[ax] - 1) hi = c + s[ax];
            else if (A.per[ax]) hi = c - (long long)(n[ax] - 1) * s[ax];
            if (hi >= 0) off += A.P[ax][hi] * x[hi];
        }
        const double v = A.diag[c] * x[c] - A.scale * off;
        y[c] = v;
        d1 += w1[c] * v;
        if (TWO) d2 += v * v;
    }
    const double s1 = block_sum<LIN_BLOCK>(d1);
    if (threadIdx.x == 0) partials[blockIdx.x] = s1;
    if (TWO) {
        const double s2 = block_sum<LIN_BLOCK>(d2);
        if (threadIdx.x == 0) partials[gridDim.x + blockIdx.x] = s2;
    }
}

// r = b, rh = b, x = 0; partial r.r
__global__ void __launch_bounds__(LIN_BLOCK) k_bicg_init(long long N, const double* __restrict__ b,
                                                         double* __restrict__ r,
                                                         double* __restrict__ rh,
                                                         double* __restrict__ x,
                                                         double* __restrict__ partials) {
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < N;
         c += (long long)gridDim.x * LIN_BLOCK) {
        const double v = b[c];
        r[c] = v;
        rh[c] = v;
        x[c] = 0.0;
        acc += v * v;
    }
    const double s = block_sum<LIN_BLOCK>(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// p = r + beta (p - omega v); first: p = r.  first < 0: decided on the device, p = r at the
// loop's first iteration and after a restart, when also the shadow vector becomes rh = r
__global__ void __launch_bounds__(LIN_BLOCK) k_bicg_p(long long N, const double* __restrict__ scal,
                                                      const double* __restrict__ r,
                                                      const double* __restrict__ v,
                                                      double* __restrict__ p, int first,
                                                      double* __restrict__ rh) {
    const double beta = scal[S_BETA], omega = scal[S_OMEGA];
    bool restart = false;
    if (first < 0) {
        restart = scal[S_RST] != 0.0;
        first = scal[S_ITS] == 0.0 || restart;
    }
    for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < N;
         c += (long long)gridDim.x * LIN_BLOCK) {
        const double rc = r[c];
        p[c] = first ? rc : rc + beta * (p[c] - omega * v[c]);
        if (restart && rh) rh[c] = rc;
    }
}

// s = r - alpha v; partial s.s
__global__ void __launch_bounds__(LIN_BLOCK) k_bicg_s(long long N, const double* __restrict__ scal,
                                                      const double* __restrict__ r,
                                                      const double* __restrict__ v,
                                                      double* __restrict__ s,
                                                      double* __restrict__ partials) {
    const double alpha = scal[S_ALPHA];
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < N;
         c += (long long)gridDim.x * LIN_BLOCK) {
        const double sv = r[c] - alpha * v[c];
        s[c] = sv;
        acc += sv * sv;
    }
    const double t = block_sum<LIN_BLOCK>(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// x += alpha ph + omega sh; r = s - omega t; partials r.r then rh.r
__global__ void __launch_bounds__(LIN_BLOCK) k_bicg_xr(long long N, const double* __restrict__ scal,
                                                       double* __restrict__ x,
                                                       const double* __restrict__ ph,
                                                       const double* __restrict__ sh,
                                                       const double* __restrict__ s,
                                                       const double* __restrict__ t,
                                                       double* __restrict__ r,
                                                       const double* __restrict__ rh,
                                                       double* __restrict__ partials) {
    const double alpha = scal[S_ALPHA], omega = scal[S_OMEGA];
    double rr = 0.0, rhr = 0.0;
    for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < N;
         c += (long long)gridDim.x * LIN_BLOCK) {
        x[c] += alpha * ph[c] + omega * sh[c];
        const double rv = s[c] - omega * t[c];
        r[c] = rv;
        rr += rv * rv;
        rhr += rh[c] * rv;
    }
    const double a1 = block_sum<LIN_BLOCK>(rr);
    if (threadIdx.x == 0) partials[blockIdx.x] = a1;
    const double a2 = block_sum<LIN_BLOCK>(rhr);
    if (threadIdx.x == 0) partials[gridDim.x + blockIdx.x] = a2;
}

// x += scal[slot] p
__global__ void __launch_bounds__(LIN_BLOCK) k_axpy(long long N, const double* __restrict__ scal,
                                                    int slot, const double* __restrict__ p,
                                                    double* __restrict__ x) {
    const double a = scal[slot];
    for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < N;
         c += (long long)gridDim.x * LIN_BLOCK)
        x[c] += a * p[c];
}

// x / r update of the device-controlled loop.  Converged at the middle of the iteration
// (S_HALF): x += alpha ph, r untouched.  Otherwise, unless a breakdown ended the iteration:
// x += alpha ph + omega sh, r = s - omega t, partials r.r then rh.r (zeros when skipped)
__global__ void __launch_bounds__(LIN_BLOCK) k_bicg_xr_loop(long long N,
                                                            const double* __restrict__ scal,
                                                            double* __restrict__ x,
                                                            const double* __restrict__ ph,
                                                            const double* __restrict__ sh,
                                                            const double* __restrict__ s,
                                                            const double* __restrict__ t,
                                                            double* __restrict__ r,
                                                            const double* __restrict__ rh,
                                                            double* __restrict__ partials) {
    const double alpha = scal[S_ALPHA], omega = scal[S_OMEGA];
    const bool half = scal[S_HALF] != 0.0;
    const bool none = !half && scal[S_DONE] != 0.0;
    double rr = 0.0, rhr = 0.0;
    if (!none) {
        for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < N;
             c += (long long)gridDim.x * LIN_BLOCK) {
            if (half) {
                x[c] += alpha * ph[c];
            } else {
                x[c] += alpha * ph[c] + omega * sh[c];
                const double rv = s[c] - omega * t[c];
                r[c] = rv;
                rr += rv * rv;
                rhr += rh[c] * rv;
            }
        }
    }
    const double a1 = block_sum<LIN_BLOCK>(rr);
    if (threadIdx.x == 0) partials[blockIdx.x] = a1;
    const double a2 = block_sum<LIN_BLOCK>(rhr);
    if (threadIdx.x == 0) partials[gridDim.x + blockIdx.x] = a2;
}

// z = x widened to FP64 (a four-per-thread form measured no faster here: 0.73 of HBM in the
// step against 0.79)
__global__ void __launch_bounds__(LIN_BLOCK) k_from_f32(long long N, const float* __restrict__ x,
                                                        double* __restrict__ z,
                                                        const double* skip) {
    if (skipped(skip)) return;
    for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < N;
         c += (long long)gridDim.x * LIN_BLOCK)
        z[c] = (double)x[c];
}

__global__ void __launch_bounds__(LIN_BLOCK) k_copy(long long N, const double* __restrict__ a,
                                                    double* __restrict__ b, const double* skip) {
    if (skipped(skip)) return;
    for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < N;
         c += (long long)gridDim.x * LIN_BLOCK)
        b[c] = a[c];
}

// The reductions of the device-controlled BiCGStab loop: a fixed-order sum of the partials
// (two sets for RED_BICG_NEXT), then the loop's scalar logic, and the continue flag written to
// S_CONT and, inside a CUDA graph, to the while node's conditional handle.
//   RED_BICG_START: r.r of r = b: S_RR = S_RHO = r.r, counters cleared; done when
//                   r.r <= S_THR (or not finite: breakdown).
//   RED_BICG_SS:    s.s: converged at the middle of the iteration when s.s <= S_THR (S_HALF,
//                   S_DONE); a breakdown flagged by the alpha reduction also sets S_DONE.
//   RED_BICG_NEXT:  r.r and rh.r: beta and rho for the next iteration, S_ITS += 1, and the
//                   loop ends when converged (or S_DONE), on a breakdown, or at S_MAXIT.
//                   When r.r has not fallen below 0.81 of its best for STALL_ITS iterations,
//                   or below S_INNER times its value at the last restart, the next iteration
//                   restarts with rh = r (up to MAX_RESTARTS times; the rounding of an FP32
//                   preconditioner slowly erodes the bi-orthogonality BiCGStab relies on); a
//                   stagnation past the last restart ends the loop, and the Newton step is
//                   then that of an inexact Newton iteration.
// This kernel always runs to its end: it is what ends the loop.
__global__ void __launch_bounds__(RED_BLOCK) k_reduce_loop(const double* __restrict__ partials,
                                                           int n, double* __restrict__ scal,
                                                           int op, unsigned long long cond) {
    const bool two = op == RED_BICG_NEXT;
    double acc = 0.0, acc2 = 0.0;
    for (int q = threadIdx.x; q < n; q += RED_BLOCK) {
        acc += partials[q];
        if (two) acc2 += partials[n + q];
    }
    const double s = block_sum<RED_BLOCK>(acc);
    const double s2 = two ? block_sum<RED_BLOCK>(acc2) : 0.0;
    if (threadIdx.x != 0) return;
    int cont = 0;
    if (op == RED_BICG_START) {
        const bool fin = isfinite(s);
        scal[S_RR] = s;
        scal[S_RHO] = s;
        scal[S_ITS] = 0.0;
        scal[S_HALF] = 0.0;
        scal[S_BREAK] = fin ? 0.0 : 1.0;
        scal[S_BEST] = s;
        scal[S_BESTIT] = 0.0;
        scal[S_STALL] = 0.0;
        scal[S_RR0] = s;
        scal[S_NRST] = 0.0;
        scal[S_RST] = 0.0;
        const bool done = !(s > scal[S_THR]) || !fin || !(scal[S_MAXIT] >= 1.0);
        scal[S_DONE] = done ? 1.0 : 0.0;
        cont = !done;
    } else if (op == RED_BICG_SS) {
        scal[S_SS] = s;
        if (!isfinite(s)) {
            scal[S_BREAK] = 1.0;
            scal[S_DONE] = 1.0;
        } else if (scal[S_BREAK] != 0.0) {
            scal[S_DONE] = 1.0;
        } else if (!(s > scal[S_THR])) {
            scal[S_HALF] = 1.0;
            scal[S_DONE] = 1.0;
        }
        return;                                    // no loop decision here
    } else {                                       // RED_BICG_NEXT
        const double its = scal[S_ITS] + 1.0;
        scal[S_ITS] = its;
        if (scal[S_DONE] != 0.0) {
            cont = 0;
        } else {
            const double rho = s2;
            scal[S_RR] = s;
            scal[S_BETA] = (rho / scal[S_RHO]) * (scal[S_ALPHA] / scal[S_OMEGA]);
            scal[S_RHO] = rho;
            const bool brk = !isfinite(s) || !(rho != 0.0) || scal[S_BREAK] != 0.0;
            if (brk) scal[S_BREAK] = 1.0;
            const bool conv = !(s > scal[S_THR]);
            if (s < 0.81 * scal[S_BEST]) {
                scal[S_BEST] = s;
                scal[S_BESTIT] = its;
            }
            bool stall = its - scal[S_BESTIT] >= (double)STALL_ITS;
            const bool inner = scal[S_INNER] > 0.0 && !(s > scal[S_INNER] * scal[S_RR0]);
            if (!conv && !brk && (stall || inner) && scal[S_NRST] < (double)MAX_RESTARTS) {
                // restart from the current x and r: fresh shadow vector rh = r, rho = r.r
                scal[S_RST] = 1.0;
                scal[S_NRST] += 1.0;
                scal[S_RR0] = s;
                scal[S_RHO] = s;
                scal[S_BEST] = s;
                scal[S_BESTIT] = its;
                stall = false;
            }
            if (stall && !conv) scal[S_STALL] = 1.0;
            // (written so that a cap that is not a number also ends the loop)
            cont = !(conv || brk || stall) && its < scal[S_MAXIT] && its < 1e6;
        }
    }
    scal[S_CONT] = cont ? 1.0 : 0.0;
    if (cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, cont ? 1u : 0u);
}

// ---------------------------------------------------------------------------------------------
// multigrid kernels (templated on the level precision)

// weighted Jacobi with wid = omega / diag: first sweep from x = 0: x_out = wid b; else
// x_out = x_in + omega (b - A x_in) / diag, written as (1 - omega) x_in + wid (b + scale off)
template <typename T>
__global__ void __launch_bounds__(LIN_BLOCK) k_mg_smooth(const Op<T> A, const T* __restrict__ b,
                                                         const T* __restrict__ xin,
                                                         T* __restrict__ xout, T omega,
                                                         int first) {
    if (skipped(A.skip)) return;
    for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < A.N;
         c += (long long)gridDim.x * LIN_BLOCK) {
        const T wi = A.wid[c];
        if (first) {
            xout[c] = wi * b[c];
        } else {
            int i, j, k;
            coords3(A, c, i, j, k);
            const T off = off_row(A, xin, c, i, j, k);
            xout[c] = jacobi_update(xin[c], b[c], wi, A.scale, off, omega);
        }
    }
}

// the first sweep of a cycle, from x = 0: x = (omega / diag) b, 16 bytes per thread (N a
// multiple of 16 / sizeof(T), 16-byte aligned arrays; the launcher checks)
template <typename T>
__global__ void __launch_bounds__(LIN_BLOCK) k_mg_smooth_first_vec(long long N,
                                                                   const T* __restrict__ wid,
                                                                   const T* __restrict__ b,
                                                                   T* __restrict__ xout,
                                                                   const double* skip) {
    if (skipped(skip)) return;
    using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    const long long NV = N * (long long)sizeof(T) / 16;
    for (long long q = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; q < NV;
         q += (long long)gridDim.x * LIN_BLOCK) {
        const VT w = __ldg(reinterpret_cast<const VT*>(wid) + q);
        const VT bb = __ldg(reinterpret_cast<const VT*>(b) + q);
        VT o;
        o.x = w.x * bb.x; o.y = w.y * bb.y;
        if constexpr (sizeof(T) == 4) { o.z = w.z * bb.z; o.w = w.w * bb.w; }
        reinterpret_cast<VT*>(xout)[q] = o;
    }
}

// Weighted-Jacobi sweep marching along z: a thread owns one (i, j) column and ZM consecutive
// planes, so the x values of the planes above and below and the z-face coefficient shared by
// two planes stay in registers, and the x / y neighbour offsets are computed once.  The
// arithmetic is that of k_mg_smooth term for term (the same products summed in the same
// order), so the result is identical.  ZM = 2: every load of both planes is issued before the
// first use within 56 registers, four blocks per SM; measured at 256^3 (FP32, both couplings
// per face), 0.91 of the HBM copy bandwidth against 0.61 for ZM = 8 (whose 104 loads do not fit
// the register budget and were issued in dependent groups) and 0.78 for one cell per thread.
constexpr int ZM = 2;
template <typename T>
__global__ void __launch_bounds__(LIN_BLOCK) k_mg_smooth_zm(const Op<T> A, const T* __restrict__ b,
                                                            const T* __restrict__ xin,
                                                            T* __restrict__ xout, T omega) {
    if (skipped(A.skip)) return;
    const long long nxy = (long long)A.nx * A.ny;
    const long long col = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x;
    if (col >= nxy) return;
    const int k0 = blockIdx.y * ZM;
    const unsigned jj = fdiv((unsigned)col, A.fd_nx);
    const int i = (int)((unsigned)col - jj * A.fd_nx.d), j = (int)jj;
    // x and y neighbour offsets (a zero-flux lower face carries W = 0 and reads the far side)
    const long long dlo0 = i > 0 ? -1 : (long long)(A.nx - 1);
    const bool hhi0 = i < A.nx - 1 || A.per[0];
    const long long dhi0 = i < A.nx - 1 ? 1 : -(long long)(A.nx - 1);
    const long long dlo1 = j > 0 ? -(long long)A.nx : (long long)(A.ny - 1) * A.nx;
    const bool hhi1 = j < A.ny - 1 || A.per[1];
    const long long dhi1 = j < A.ny - 1 ? (long long)A.nx : -(long long)(A.ny - 1) * A.nx;
    const int nz = A.nz;
    // read-only operator arrays through non-aliasing pointers, so that the loads of later
    // planes may be issued before the stores of earlier ones
    const T* __restrict__ W0 = A.W[0];
    const T* __restrict__ W1 = A.W[1];
    const T* __restrict__ W2 = A.W[2];
    const T* __restrict__ P0 = A.Wp[0];
    const T* __restrict__ P1 = A.Wp[1];
    const T* __restrict__ P2 = A.Wp[2];
    const T* __restrict__ wd = A.wid;
    // z: plane below k0 (the far side when k0 = 0: W = 0 there unless periodic).  All loads of
    // the ZM planes are issued first (registers), then the planes are computed in order;
    // the launcher uses this kernel only when ZM divides nz.
    const long long c0 = col + (long long)k0 * nxy;
    const long long ctop = k0 + ZM < nz ? c0 + (long long)ZM * nxy : col;   // plane above
    // wz: the lower-face coupling of each plane's row; pz: the coupling of each plane's row to
    // the plane above (Wp of the face above; the same numbers as wz[kk + 1] when symmetric)
    T xz[ZM + 2], wz[ZM], pz[ZM], w0l[ZM], w0h[ZM], w1l[ZM], w1h[ZM], x0l[ZM], x0h[ZM], x1l[ZM],
        x1h[ZM], dd[ZM], bb[ZM];
    xz[0] = __ldg(xin + (k0 > 0 ? c0 - nxy : col + (long long)(nz - 1) * nxy));
    xz[ZM + 1] = __ldg(xin + ctop);
#pragma unroll
    for (int kk = 0; kk < ZM; ++kk) {
        const long long c = c0 + (long long)kk * nxy;
        const long long cu = kk + 1 < ZM ? c + nxy : ctop;
        xz[kk + 1] = __ldg(xin + c);
        wz[kk] = __ldg(W2 + c);
        pz[kk] = __ldg(P2 + cu);
        w0l[kk] = __ldg(W0 + c);
        x0l[kk] = __ldg(xin + c + dlo0);
        w0h[kk] = hhi0 ? __ldg(P0 + c + dhi0) : T(0);
        x0h[kk] = hhi0 ? __ldg(xin + c + dhi0) : T(0);
        w1l[kk] = __ldg(W1 + c);
        x1l[kk] = __ldg(xin + c + dlo1);
        w1h[kk] = hhi1 ? __ldg(P1 + c + dhi1) : T(0);
        x1h[kk] = hhi1 ? __ldg(xin + c + dhi1) : T(0);
        dd[kk] = __ldg(wd + c);
        bb[kk] = __ldg(b + c);
    }
#pragma unroll
    for (int kk = 0; kk < ZM; ++kk) {
        const bool hz = k0 + kk < nz - 1 || A.per[2];
        T off = T(0);
        off += w0l[kk] * x0l[kk];
        if (hhi0) off += w0h[kk] * x0h[kk];
        off += w1l[kk] * x1l[kk];
        if (hhi1) off += w1h[kk] * x1h[kk];
        off += wz[kk] * xz[kk];
        if (hz) off += pz[kk] * xz[kk + 2];
        xout[c0 + (long long)kk * nxy] = jacobi_update(xz[kk + 1], bb[kk], dd[kk], A.scale, off, omega);
    }
}

// The same FP32 sweep with its rows staged in shared memory by bulk asynchronous copies.  A
// CTA owns one grid row (j) of every plane of a z-slab of ZB planes, one thread per x cell.
// For each plane it needs 12 contiguous rows of nx floats: x at (j, k), (j-1, k), (j+1, k),
// (j, k+1); b, omega / diag and the lower-face couplings W0, W1, W2 and P0 at (j, k); P1 at
// (j+1, k); P2 at (j, k+1).  One elected thread issues them as cp.async.bulk copies into a
// ring of BS stages, each completing on its stage's mbarrier; the CTA computes plane k from
// shared memory while the copies of the next planes are in flight.  Rows whose neighbour
// does not exist (zero-flux faces) are fetched from a valid row and not used, as in
// k_mg_smooth_zm, whose products and sums this kernel repeats term for term.  Requirements
// (checked by the launcher): nx a multiple of 4 and at most BULK_MAX_NX, 16-byte aligned
// arrays, nz a multiple of ZB.  Each wait on a stage is bounded: after BULK_SPIN tries the
// kernel records the plane in *err, waits (bounded) for its own copies once more, and
// returns.
constexpr int BULK_ROWS = 12;
constexpr int BULK_STAGES = 3;
constexpr int BULK_ZB = 16;
constexpr int BULK_MAX_NX = 512;
constexpr long long BULK_SPIN = 1LL << 24;

// set to 1 by a staged sweep whose wait on a stage timed out
__device__ int g_bulk_wait_error = 0;
static int* g_bulk_err_ptr = nullptr;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}" 
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase `parity` of a stage barrier; false on timeout
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
    for (long long t = 0; t < BULK_SPIN; ++t)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__global__ void __launch_bounds__(BULK_MAX_NX) k_mg_smooth_bulk(const Op<float> A,
                                                                const float* __restrict__ b,
                                                                const float* __restrict__ xin,
                                                                float* __restrict__ xout,
                                                                float omega, int* err) {
    if (skipped(A.skip)) return;
    extern __shared__ __align__(128) float rows[];          // [BULK_STAGES][BULK_ROWS][nx]
    __shared__ __align__(8) unsigned long long bar[BULK_STAGES];
    const int nx = A.nx, ny = A.ny, nz = A.nz;
    const int i = threadIdx.x;
    const int j = blockIdx.x;
    const int k0 = blockIdx.y * BULK_ZB;
    const long long nxy = (long long)nx * ny;
    const int jm = j > 0 ? j - 1 : ny - 1;
    const int jp = j < ny - 1 ? j + 1 : 0;
    const bool hhi0 = i < nx - 1 || A.per[0];
    const bool hhi1 = j < ny - 1 || A.per[1];
    const unsigned row_bytes = (unsigned)nx * 4u;
    auto stage_row = [&](int st, int r) { return rows + ((long long)st * BULK_ROWS + r) * nx; };
    // the copies of plane k into stage st (one elected thread)
    auto issue = [&](int k, int st) {
        const int ku = k + 1 < nz ? k + 1 : 0;
        const long long c = (long long)j * nx + (long long)k * nxy;
        const long long cm = (long long)jm * nx + (long long)k * nxy;
        const long long cp = (long long)jp * nx + (long long)k * nxy;
        const long long cu = (long long)j * nx + (long long)ku * nxy;
        const float* src[BULK_ROWS] = {xin + c, xin + cm, xin + cp, xin + cu, b + c, A.wid + c,
                                       A.W[0] + c, A.W[1] + c, A.W[2] + c, A.Wp[0] + c,
                                       A.Wp[1] + cp, A.Wp[2] + cu};
        mbar_expect_tx(&bar[st], row_bytes * BULK_ROWS);
#pragma unroll
        for (int r = 0; r < BULK_ROWS; ++r) bulk_g2s(stage_row(st, r), src[r], row_bytes, &bar[st]);
    };
    if (i == 0) {
#pragma unroll
        for (int st = 0; st < BULK_STAGES; ++st) mbar_init(&bar[st], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (i == 0) {
#pragma unroll
        for (int st = 0; st < BULK_STAGES; ++st)
            if (st < BULK_ZB) issue(k0 + st, st);
    }
    // x of the plane below the first one (the far side when k0 = 0: W = 0 there unless periodic)
    float xlo = i < nx ? __ldg(xin + (long long)j * nx + (long long)(k0 > 0 ? k0 - 1 : nz - 1) * nxy + i)
                       : 0.f;
    bool ok = true;
    for (int kk = 0; kk < BULK_ZB; ++kk) {
        const int st = kk % BULK_STAGES;
        const unsigned parity = (unsigned)((kk / BULK_STAGES) & 1);
        if (!mbar_wait(&bar[st], parity)) { ok = false; break; }
        const int k = k0 + kk;
        float xcen = 0.f;
        if (i < nx) {
            const float* XC = stage_row(st, 0);
            const float* XM = stage_row(st, 1);
            const float* XP = stage_row(st, 2);
            const float* XU = stage_row(st, 3);
            const float* BB = stage_row(st, 4);
            const float* WD = stage_row(st, 5);
            const float* R0 = stage_row(st, 6);
            const float* R1 = stage_row(st, 7);
            const float* R2 = stage_row(st, 8);
            const float* Q0 = stage_row(st, 9);
            const float* Q1 = stage_row(st, 10);
            const float* Q2 = stage_row(st, 11);
            const int il = i > 0 ? i - 1 : nx - 1;
            const int ih = i < nx - 1 ? i + 1 : 0;
            const bool hz = k < nz - 1 || A.per[2];
            xcen = XC[i];
            float off = 0.f;
            off += R0[i] * XC[il];
            if (hhi0) off += Q0[ih] * XC[ih];
            off += R1[i] * XM[i];
            if (hhi1) off += Q1[i] * XP[i];
            off += R2[i] * xlo;
            if (hz) off += Q2[i] * XU[i];
            xout[(long long)j * nx + (long long)k * nxy + i] =
                jacobi_update(xcen, BB[i], WD[i], A.scale, off, omega);
        }
        xlo = xcen;
        __syncthreads();                                    // stage st is free again
        if (i == 0 && kk + BULK_STAGES < BULK_ZB) issue(k0 + kk + BULK_STAGES, st);
    }
    if (!ok) {
        if (i == 0) atomicExch(err, 1);
        // the copies this CTA issued may still land: wait for them once more, bounded
        for (int st = 0; st < BULK_STAGES; ++st) mbar_wait(&bar[st], 0u);
    }
}

cudaError_t linear_kernels_init() {
    if (g_bulk_err_ptr) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_mg_smooth_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         BULK_STAGES * BULK_ROWS * BULK_MAX_NX * (int)sizeof(float));
    void* p = nullptr;
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&p, g_bulk_wait_error);
    if (e == cudaSuccess) g_bulk_err_ptr = static_cast<int*>(p);
    return e;
}
cudaError_t bulk_wait_flag_read(int* host, cudaStream_t st) {
    return cudaMemcpyFromSymbolAsync(host, g_bulk_wait_error, sizeof(int), 0, cudaMemcpyDeviceToHost, st);
}
cudaError_t bulk_wait_flag_clear(cudaStream_t st) {
    static const int zero = 0;
    return cudaMemcpyToSymbolAsync(g_bulk_wait_error, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st);
}

// all Jacobi sweeps of the coarsest level in one CTA: the same arithmetic as that many
// k_mg_smooth launches (first sweep from x = 0 into x, then x and xt alternate), with a block
// barrier in place of each kernel boundary
constexpr int COARSE_BLOCK = 1024;
template <typename T>
__global__ void __launch_bounds__(COARSE_BLOCK) k_mg_coarse(const Op<T> A, const T* __restrict__ b,
                                                            T* x, T* xt, T omega, int sweeps) {
    if (skipped(A.skip)) return;
    T* buf[2] = {x, xt};
    for (int s = 0; s < sweeps; ++s) {
        const T* xin = buf[(s + 1) & 1];
        T* xout = buf[s & 1];
        for (long long c = threadIdx.x; c < A.N; c += COARSE_BLOCK) {
            const T wi = A.wid[c];
            if (s == 0) {
                xout[c] = wi * b[c];
            } else {
                int i, j, k;
                coords3(A, c, i, j, k);
                const T off = off_row(A, xin, c, i, j, k);
                xout[c] = jacobi_update(xin[c], b[c], wi, A.scale, off, omega);
            }
        }
        __syncthreads();
    }
}

// coarse right-hand side: (sum over the children of the fine residual b - A x) / 8, the
// transpose of the injection prolongation scaled by 1/8 (a parent with fewer than 8 children,
// at an odd extent, keeps the factor, so that the cycle stays symmetric).
//
// FP64 and symmetric: with (A x)_c = loc_c x_c + scale sum_faces W (x_c - x_nb), the faces
// between two children of the parent cancel in the sum, so only the faces to cells outside the
// parent are evaluated; this halves the FP64 arithmetic that bounds the FP64 instance.  (For a
// non-symmetric operator the two rows of an inner face carry W and Wp, which do not cancel.)
// Otherwise the residual of each child from its full row, which for FP32 also measured faster
// at 256^3 (16.2 against 18.8 ms per step, where the outside-face form took FP64 from 48.0 down
// to 41.9 ms).
template <typename T>
__global__ void __launch_bounds__(LIN_BLOCK) k_mg_restrict(const Op<T> A, const T* __restrict__ b,
                                                           const T* __restrict__ x, int cnx,
                                                           int cny, int cnz, FastDiv fcx,
                                                           FastDiv fcxy, T* __restrict__ bc) {
    if (skipped(A.skip)) return;
    const long long Nc = (long long)cnx * cny * cnz;
    const long long sz = (long long)A.nx * A.ny;
    const int n[3] = {A.nx, A.ny, A.nz};
    const long long s[3] = {1, A.nx, sz};
    for (long long cc = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; cc < Nc;
         cc += (long long)gridDim.x * LIN_BLOCK) {
        int I, J, K;
        coords_fd(cc, fcx, fcxy, I, J, K);
        T acc = T(0);
        const bool inner_cancel = sizeof(T) == 8 && A.loc && A.Wp[0] == A.W[0];
        if (inner_cancel) {
#pragma unroll
            for (int dk = 0; dk < 2; ++dk) {
#pragma unroll
                for (int dj = 0; dj < 2; ++dj) {
#pragma unroll
                    for (int di = 0; di < 2; ++di) {
                        const int q[3] = {2 * I + di, 2 * J + dj, 2 * K + dk};
                        if (q[0] >= n[0] || q[1] >= n[1] || q[2] >= n[2]) continue;  // odd end
                        const int d[3] = {di, dj, dk};
                        const long long c = q[0] + (long long)A.nx * (q[1] + (long long)A.ny * q[2]);
                        const T xc = x[c];
                        T fl = T(0);
#pragma unroll
                        for (int ax = 0; ax < 3; ++ax) {
                            if (d[ax] == 0) {         // lower face: the neighbour is outside
                                const long long lo = q[ax] > 0 ? c - s[ax]
                                                               : c + (long long)(n[ax] - 1) * s[ax];
                                fl += A.W[ax][c] * (xc - x[lo]);   // W = 0 on zero-flux faces
                            }
                            // upper face: outside unless it leads to the sibling d = 1
                            if (d[ax] == 1 || q[ax] + 1 >= n[ax]) {
                                long long hi = -1;
                                if (q[ax] < n[ax] - 1) hi = c + s[ax];
                                else if (A.per[ax]) hi = c - (long long)(n[ax] - 1) * s[ax];
                                if (hi >= 0) fl += A.W[ax][hi] * (xc - x[hi]);
                            }
                        }
                        acc += b[c] - A.loc[c] * xc - A.scale * fl;
                    }
                }
            }
        } else {
            for (int dk = 0; dk < 2; ++dk) {
                const int k = 2 * K + dk;
                if (k >= A.nz) continue;
                for (int dj = 0; dj < 2; ++dj) {
                    const int j = 2 * J + dj;
                    if (j >= A.ny) continue;
                    for (int di = 0; di < 2; ++di) {
                        const int i = 2 * I + di;
                        if (i >= A.nx) continue;
                        const long long c = i + (long long)A.nx * (j + (long long)A.ny * k);
                        acc += b[c] - apply_row(A, x, c, i, j, k, x[c]);
                    }
                }
            }
        }
        bc[cc] = acc * T(0.125);
    }
}

// x_f += x_c(parent), 16 bytes of fine cells per thread along x (4 FP32 or 2 FP64 cells, whose
// parents are 2 or 1 consecutive coarse cells); needs nx a multiple of 4 (FP32) or 2 (FP64) and
// 16-byte aligned rows, which the launcher checks.  fx, fxy divide by nx / V and nx ny / V.
template <typename T>
__global__ void __launch_bounds__(LIN_BLOCK) k_mg_prolong_vec(int nx, int ny, int nz, int cnx,
                                                              int cny, FastDiv fx, FastDiv fxy,
                                                              const T* __restrict__ xc,
                                                              T* __restrict__ xf,
                                                              const double* skip) {
    if (skipped(skip)) return;
    constexpr int V = 16 / (int)sizeof(T);
    using VT = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    const long long NV = (long long)nx * ny * nz / V;
    for (long long q = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; q < NV;
         q += (long long)gridDim.x * LIN_BLOCK) {
        int iv, j, k;
        coords_fd(q, fx, fxy, iv, j, k);
        const T* pc = xc + (long long)(V / 2) * iv + (long long)cnx * ((j >> 1) + (long long)cny * (k >> 1));
        VT v = reinterpret_cast<VT*>(xf)[q];
        if constexpr (sizeof(T) == 4) {
            const float2 pp = *reinterpret_cast<const float2*>(pc);
            v.x += pp.x; v.y += pp.x; v.z += pp.y; v.w += pp.y;
        } else {
            const double pp = *pc;
            v.x += pp; v.y += pp;
        }
        reinterpret_cast<VT*>(xf)[q] = v;
    }
}

// x_f += x_c(parent)
template <typename T>
__global__ void __launch_bounds__(LIN_BLOCK) k_mg_prolong(int nx, int ny, int nz, int cnx, int cny,
                                                          FastDiv fx, FastDiv fxy,
                                                          const T* __restrict__ xc,
                                                          T* __restrict__ xf,
                                                          const double* skip) {
    if (skipped(skip)) return;
    const long long N = (long long)nx * ny * nz;
    for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < N;
         c += (long long)gridDim.x * LIN_BLOCK) {
        int i, j, k;
        coords_fd(c, fx, fxy, i, j, k);
        xf[c] += xc[(i >> 1) + (long long)cnx * ((j >> 1) + (long long)cny * (k >> 1))];
    }
}

// Coarse operator by re-discretisation: local diagonal = mean of the children's local
// diagonals (diag - scale * the six couplings of their rows); each face array of the coarse
// cell's lower face = (mean of that array over the existing fine lower faces of its first-layer
// children) / 4, W from W and, for a non-symmetric operator, Wp from Wp (wpc null: symmetric).
// Writes diag_c = local part only; k_mg_diag_faces adds the row's couplings.
template <typename TF, typename TC>
__global__ void __launch_bounds__(LIN_BLOCK) k_mg_coarsen(const Op<TF> A, int cnx, int cny,
                                                          int cnz, TC* __restrict__ dc,
                                                          TC* __restrict__ wcx,
                                                          TC* __restrict__ wcy,
                                                          TC* __restrict__ wcz,
                                                          TC* __restrict__ wpcx,
                                                          TC* __restrict__ wpcy,
                                                          TC* __restrict__ wpcz) {
    const long long Nc = (long long)cnx * cny * cnz;
    const long long sz = (long long)A.nx * A.ny;
    for (long long cc = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; cc < Nc;
         cc += (long long)gridDim.x * LIN_BLOCK) {
        const int K = (int)(cc / ((long long)cnx * cny));
        const long long rem = cc - (long long)K * cnx * cny;
        const int J = (int)(rem / cnx), I = (int)(rem - (long long)J * cnx);
        double dl = 0.0, wl[3] = {0.0, 0.0, 0.0}, wp[3] = {0.0, 0.0, 0.0};
        int cnt = 0, nf[3] = {0, 0, 0};
        for (int dk = 0; dk < 2; ++dk) {
            const int k = 2 * K + dk;
            if (k >= A.nz) continue;
            for (int dj = 0; dj < 2; ++dj) {
                const int j = 2 * J + dj;
                if (j >= A.ny) continue;
                for (int di = 0; di < 2; ++di) {
                    const int i = 2 * I + di;
                    if (i >= A.nx) continue;
                    const long long c = i + (long long)A.nx * (j + (long long)A.ny * k);
                    // the six couplings of the child's row
                    double fsum = 0.0;
                    const int q[3] = {i, j, k};
                    const int n[3] = {A.nx, A.ny, A.nz};
                    const long long s[3] = {1, A.nx, sz};
                    const int d[3] = {di, dj, dk};
#pragma unroll
                    for (int ax = 0; ax < 3; ++ax) {
                        fsum += (double)A.W[ax][c];
                        if (q[ax] < n[ax] - 1) fsum += (double)A.Wp[ax][c + s[ax]];
                        else if (A.per[ax]) fsum += (double)A.Wp[ax][c - (long long)(n[ax] - 1) * s[ax]];
                        if (d[ax] == 0) {
                            wl[ax] += (double)A.W[ax][c];
                            wp[ax] += (double)A.Wp[ax][c];
                            ++nf[ax];
                        }
                    }
                    dl += (double)A.diag[c] - (double)A.scale * fsum;
                    ++cnt;
                }
            }
        }
        const double sc = (double)A.scale * 0.25;
        dc[cc] = (TC)(dl / cnt);
        wcx[cc] = (TC)(sc * wl[0] / nf[0]);
        wcy[cc] = (TC)(sc * wl[1] / nf[1]);
        wcz[cc] = (TC)(sc * wl[2] / nf[2]);
        if (wpcx) {
            wpcx[cc] = (TC)(sc * wp[0] / nf[0]);
            wpcy[cc] = (TC)(sc * wp[1] / nf[1]);
            wpcz[cc] = (TC)(sc * wp[2] / nf[2]);
        }
    }
}

// diag += sum of the six couplings of the row (scale 1 on coarse levels)
template <typename T>
__global__ void __launch_bounds__(LIN_BLOCK) k_mg_diag_faces(Op<T> A, T* __restrict__ diag) {
    const long long sz = (long long)A.nx * A.ny;
    for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < A.N;
         c += (long long)gridDim.x * LIN_BLOCK) {
        int i, j, k;
        coords3(A, c, i, j, k);
        const int q[3] = {i, j, k};
        const int n[3] = {A.nx, A.ny, A.nz};
        const long long s[3] = {1, A.nx, sz};
        T f = T(0);
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            f += A.W[ax][c];
            if (q[ax] < n[ax] - 1) f += A.Wp[ax][c + s[ax]];
            else if (A.per[ax]) f += A.Wp[ax][c - (long long)(n[ax] - 1) * s[ax]];
        }
        diag[c] += f;
    }
}

// FP32 copy of the finest operator with the scale folded into the faces (W and, when the
// operator is non-symmetric, Wp)
__global__ void __launch_bounds__(LIN_BLOCK) k_cast_op(const Op<double> A, float* __restrict__ d,
                                                       float* __restrict__ wx,
                                                       float* __restrict__ wy,
                                                       float* __restrict__ wz,
                                                       float* __restrict__ px,
                                                       float* __restrict__ py,
                                                       float* __restrict__ pz) {
    for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < A.N;
         c += (long long)gridDim.x * LIN_BLOCK) {
        d[c] = (float)A.diag[c];
        wx[c] = (float)(A.scale * A.W[0][c]);
        wy[c] = (float)(A.scale * A.W[1][c]);
        wz[c] = (float)(A.scale * A.W[2][c]);
        if (px) {
            px[c] = (float)(A.scale * A.Wp[0][c]);
            py[c] = (float)(A.scale * A.Wp[1][c]);
            pz[c] = (float)(A.scale * A.Wp[2][c]);
        }
    }
}

// wid = omega / diag and, where loc is given, loc = diag - scale * (sum of the six couplings of
// the row), in TF
template <typename TF, typename TO>
__global__ void __launch_bounds__(LIN_BLOCK) k_mg_level_prep(const Op<TF> A, double omega,
                                                             TO* __restrict__ wid,
                                                             TO* __restrict__ loc) {
    const long long sz = (long long)A.nx * A.ny;
    for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < A.N;
         c += (long long)gridDim.x * LIN_BLOCK) {
        const TF d = A.diag[c];
        wid[c] = (TO)((TF)omega / d);
        if (loc) {
            int i, j, k;
            coords3(A, c, i, j, k);
            const int q[3] = {i, j, k};
            const int n[3] = {A.nx, A.ny, A.nz};
            const long long s[3] = {1, A.nx, sz};
            TF f = TF(0);
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                f += A.W[ax][c];
                if (q[ax] < n[ax] - 1) f += A.Wp[ax][c + s[ax]];
                else if (A.per[ax]) f += A.Wp[ax][c - (long long)(n[ax] - 1) * s[ax]];
            }
            loc[c] = (TO)(d - A.scale * f);
        }
    }
}

template <bool VEC>
__global__ void __launch_bounds__(LIN_BLOCK) k_to_f32(long long N, const double* __restrict__ a,
                                                      float* __restrict__ b, const double* skip) {
    if (skipped(skip)) return;
    long long done = 0;
    if (VEC) {
        const long long N4 = N / 4;
        for (long long q = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; q < N4;
             q += (long long)gridDim.x * LIN_BLOCK) {
            const double2 u = reinterpret_cast<const double2*>(a)[2 * q];
            const double2 v = reinterpret_cast<const double2*>(a)[2 * q + 1];
            reinterpret_cast<float4*>(b)[q] = make_float4((float)u.x, (float)u.y, (float)v.x, (float)v.y);
        }
        done = 4 * N4;
    }
    for (long long c = done + blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < N;
         c += (long long)gridDim.x * LIN_BLOCK)
        b[c] = (float)a[c];
}

// z = x (widened); partial r.z
__global__ void __launch_bounds__(LIN_BLOCK) k_from_f32_dot(long long N, const float* __restrict__ x,
                                                            const double* __restrict__ r,
                                                            double* __restrict__ z,
                                                            double* __restrict__ partials) {
    double acc = 0.0;
    for (long long c = blockIdx.x * (long long)LIN_BLOCK + threadIdx.x; c < N;
         c += (long long)gridDim.x * LIN_BLOCK) {
        const double zv = (double)x[c];
        z[c] = zv;
        acc += r[c] * zv;
    }
    const double s = block_sum<LIN_BLOCK>(acc);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// ---------------------------------------------------------------------------------------------
// host-side launchers

LinLaunch::LinLaunch(cudaStream_t s, LaunchHook* h) : st(s), hook(h) {}

void LinLaunch::begin(const char* name) { if (hook) hook->begin(name); }
cudaError_t LinLaunch::end() {
    cudaError_t e = cudaGetLastError();
    if (hook) hook->end();
    return e;
}

cudaError_t LinLaunch::matvec_dot(const Op<double>& A, const double* p, double* q, double* part,
                                  int& nparts) {
    nparts = stream_blocks(A.N);
    begin("cg_matvec_dot");
    k_matvec_dot<<<nparts, LIN_BLOCK, 0, st>>>(A, p, q, part);
    return end();
}
cudaError_t LinLaunch::cg_xr(long long N, const double* scal, double* x, double* r,
                             const double* p, const double* q, double* part, int& nparts) {
    nparts = stream_blocks(N);
    begin("cg_update_xr");
    k_cg_xr<<<nparts, LIN_BLOCK, 0, st>>>(N, scal, x, r, p, q, part);
    return end();
}
cudaError_t LinLaunch::cg_p(long long N, const double* scal, const double* z, double* p, int first) {
    begin("cg_update_p");
    k_cg_p<<<stream_blocks(N), LIN_BLOCK, 0, st>>>(N, scal, z, p, first);
    return end();
}
cudaError_t LinLaunch::jacobi_dot(long long N, const double* r, const double* diag, double* z,
                                  double* part, int& nparts) {
    nparts = stream_blocks(N);
    begin("precond_jacobi");
    k_jacobi_dot<<<nparts, LIN_BLOCK, 0, st>>>(N, r, diag, z, part, skip);
    return end();
}
cudaError_t LinLaunch::dot(long long N, const double* a, const double* b, double* part,
                           int& nparts) {
    nparts = stream_blocks(N);
    begin("dot");
    k_dot<<<nparts, LIN_BLOCK, 0, st>>>(N, a, b, part);
    return end();
}
cudaError_t LinLaunch::cg_init(long long N, const double* b, double* r, double* x, double* part,
                               int& nparts) {
    nparts = stream_blocks(N);
    begin("cg_init");
    k_cg_init<<<nparts, LIN_BLOCK, 0, st>>>(N, b, r, x, part);
    return end();
}
cudaError_t LinLaunch::reduce(const double* part, int n, double* scal, int op, int slot) {
    begin("reduce");
    k_reduce<<<1, RED_BLOCK, 0, st>>>(part, n, scal, op, slot, skip);
    return end();
}
cudaError_t LinLaunch::reduce_loop(const double* part, int n, double* scal, int op,
                                   unsigned long long cond) {
    begin("reduce");
    k_reduce_loop<<<1, RED_BLOCK, 0, st>>>(part, n, scal, op, cond);
    return end();
}
cudaError_t LinLaunch::bicg_xr_loop(long long N, const double* scal, double* x, const double* ph,
                                    const double* sh, const double* s, const double* t,
                                    double* r, const double* rh, double* part, int& nparts) {
    nparts = stream_blocks(N);
    begin("bicg_update_xr");
    k_bicg_xr_loop<<<nparts, LIN_BLOCK, 0, st>>>(N, scal, x, ph, sh, s, t, r, rh, part);
    return end();
}
cudaError_t LinLaunch::from_f32(long long N, const float* x, double* z) {
    begin("mg_from_f32");
    k_from_f32<<<stream_blocks(N), LIN_BLOCK, 0, st>>>(N, x, z, skip);
    return end();
}
cudaError_t LinLaunch::copy(long long N, const double* a, double* b) {
    begin("copy");
    k_copy<<<stream_blocks(N), LIN_BLOCK, 0, st>>>(N, a, b, skip);
    return end();
}

cudaError_t LinLaunch::matvec_ns(const OpNS& A, const double* x, double* y, const double* w1,
                                 int two_dots, double* part, int& nparts) {
    nparts = stream_blocks(A.N);
    begin("bicg_matvec");
    OpNS B = A;
    B.skip = skip;
    if (two_dots) k_matvec_ns<true><<<nparts, LIN_BLOCK, 0, st>>>(B, x, y, w1, part);
    else k_matvec_ns<false><<<nparts, LIN_BLOCK, 0, st>>>(B, x, y, w1, part);
    return end();
}
cudaError_t LinLaunch::bicg_init(long long N, const double* b, double* r, double* rh, double* x,
                                 double* part, int& nparts) {
    nparts = stream_blocks(N);
    begin("bicg_init");
    k_bicg_init<<<nparts, LIN_BLOCK, 0, st>>>(N, b, r, rh, x, part);
    return end();
}
cudaError_t LinLaunch::bicg_p(long long N, const double* scal, const double* r, const double* v,
                              double* p, int first, double* rh) {
    begin("bicg_update_p");
    k_bicg_p<<<stream_blocks(N), LIN_BLOCK, 0, st>>>(N, scal, r, v, p, first, rh);
    return end();
}
cudaError_t LinLaunch::bicg_s(long long N, const double* scal, const double* r, const double* v,
                              double* s, double* part, int& nparts) {
    nparts = stream_blocks(N);
    begin("bicg_update_s");
    k_bicg_s<<<nparts, LIN_BLOCK, 0, st>>>(N, scal, r, v, s, part);
    return end();
}
cudaError_t LinLaunch::bicg_xr(long long N, const double* scal, double* x, const double* ph,
                               const double* sh, const double* s, const double* t, double* r,
                               const double* rh, double* part, int& nparts) {
    nparts = stream_blocks(N);
    begin("bicg_update_xr");
    k_bicg_xr<<<nparts, LIN_BLOCK, 0, st>>>(N, scal, x, ph, sh, s, t, r, rh, part);
    return end();
}
cudaError_t LinLaunch::axpy(long long N, const double* scal, int slot, const double* p, double* x) {
    begin("axpy");
    k_axpy<<<stream_blocks(N), LIN_BLOCK, 0, st>>>(N, scal, slot, p, x);
    return end();
}

template <typename T>
cudaError_t LinLaunch::smooth(const Op<T>& A, const T* b, const T* xin, T* xout, T omega,
                              int first) {
    // the finest level's sweeps get their own names (the first sweep of a cycle, from x = 0,
    // reads only b and omega / diag)
    if (A.N == fine_N && first) begin(sizeof(T) == 4 ? "mg_smooth_f32_fine_first" : "mg_smooth_f64_fine_first");
    else if (A.N == fine_N) begin(sizeof(T) == 4 ? "mg_smooth_f32_fine" : "mg_smooth_f64_fine");
    else begin(sizeof(T) == 4 ? "mg_smooth_f32" : "mg_smooth_f64");
    const long long nxy = (long long)A.nx * A.ny;
    Op<T> B = A;
    B.skip = skip;
    // (FP32 only: the FP64 sweep is bound by its FP64 arithmetic, not by load latency, and
    // its z-marching form measured slower)
    const auto al16 = [](const void* p) { return ((unsigned long long)p & 15ull) == 0; };
    // the staged sweep on large rows (measured 0.966 of HBM against 0.909 for the z-march at
    // 256^3, even at 192^3, and slower on rows of 128 whose level fits in L2)
    bool bulk_ok = false;
    if constexpr (sizeof(T) == 4) {
        bulk_ok = !first && xin != xout && g_bulk_err_ptr && A.nx % 4 == 0 && A.nx >= 256 &&
                  A.nx <= BULK_MAX_NX && A.nz % BULK_ZB == 0 && al16(xin) && al16(b) &&
                  al16(A.wid) && al16(A.W[0]) && al16(A.W[1]) && al16(A.W[2]) &&
                  al16(A.Wp[0]) && al16(A.Wp[1]) && al16(A.Wp[2]);
    }
    if (first && (A.N * (long long)sizeof(T)) % 16 == 0 && al16(A.wid) && al16(b) && al16(xout)) {
        k_mg_smooth_first_vec<T><<<stream_blocks(A.N * (long long)sizeof(T) / 16), LIN_BLOCK, 0, st>>>(
            A.N, A.wid, b, xout, skip);
    } else if (bulk_ok) {
        if constexpr (sizeof(T) == 4) {
            const size_t smem = (size_t)BULK_STAGES * BULK_ROWS * A.nx * sizeof(float);
            k_mg_smooth_bulk<<<dim3((unsigned)A.ny, (unsigned)(A.nz / BULK_ZB)),
                               (unsigned)((A.nx + 31) / 32 * 32), smem, st>>>(
                B, b, xin, xout, omega, g_bulk_err_ptr);
        }
    } else if (sizeof(T) == 4 && !first && A.nz % ZM == 0 && nxy >= 4 * LIN_BLOCK && xin != xout) {
        const dim3 g((unsigned)((nxy + LIN_BLOCK - 1) / LIN_BLOCK), (unsigned)((A.nz + ZM - 1) / ZM));
        k_mg_smooth_zm<T><<<g, LIN_BLOCK, 0, st>>>(B, b, xin, xout, omega);
    } else {
        k_mg_smooth<T><<<stream_blocks(A.N), LIN_BLOCK, 0, st>>>(B, b, xin, xout, omega, first);
    }
    return end();
}
template <typename T>
cudaError_t LinLaunch::coarse_solve(const Op<T>& A, const T* b, T* x, T* xt, T omega, int sweeps) {
    begin(sizeof(T) == 4 ? "mg_coarse_f32" : "mg_coarse_f64");
    Op<T> B = A;
    B.skip = skip;
    k_mg_coarse<T><<<1, COARSE_BLOCK, 0, st>>>(B, b, x, xt, omega, sweeps);
    return end();
}
template <typename T>
cudaError_t LinLaunch::restrict_res(const Op<T>& A, const T* b, const T* x, int cnx, int cny,
                                    int cnz, T* bc) {
    if (A.N == fine_N) begin(sizeof(T) == 4 ? "mg_restrict_f32_fine" : "mg_restrict_f64_fine");
    else begin(sizeof(T) == 4 ? "mg_restrict_f32" : "mg_restrict_f64");
    Op<T> B = A;
    B.skip = skip;
    k_mg_restrict<T><<<stream_blocks((long long)cnx * cny * cnz), LIN_BLOCK, 0, st>>>(
        B, b, x, cnx, cny, cnz, make_fastdiv((unsigned)cnx), make_fastdiv((unsigned)cnx * cny), bc);
    return end();
}
template <typename T>
cudaError_t LinLaunch::prolong(int nx, int ny, int nz, int cnx, int cny, const T* xc, T* xf) {
    if ((long long)nx * ny * nz == fine_N) begin(sizeof(T) == 4 ? "mg_prolong_f32_fine" : "mg_prolong_f64_fine");
    else begin(sizeof(T) == 4 ? "mg_prolong_f32" : "mg_prolong_f64");
    constexpr int V = 16 / (int)sizeof(T);
    const long long NV = (long long)nx * ny * nz / V;
    // the vector form: whole 16-byte groups of fine cells along x, their parents at an offset
    // of V / 2 per group (cnx = nx / 2 is then a multiple of V / 2), aligned rows
    if (nx % V == 0 && cnx * 2 == nx && ((unsigned long long)xf & 15ull) == 0 &&
        ((unsigned long long)xc & (sizeof(T) * V / 2 - 1)) == 0) {
        k_mg_prolong_vec<T><<<stream_blocks(NV), LIN_BLOCK, 0, st>>>(
            nx, ny, nz, cnx, cny, make_fastdiv((unsigned)(nx / V)), make_fastdiv((unsigned)(nx / V) * ny),
            xc, xf, skip);
    } else {
        k_mg_prolong<T><<<stream_blocks((long long)nx * ny * nz), LIN_BLOCK, 0, st>>>(
            nx, ny, nz, cnx, cny, make_fastdiv((unsigned)nx), make_fastdiv((unsigned)nx * ny), xc,
            xf, skip);
    }
    return end();
}
template <typename TF, typename TC>
cudaError_t LinLaunch::coarsen(const Op<TF>& A, int cnx, int cny, int cnz, TC* dc, TC* const* wc,
                               TC* const* wpc) {
    begin("mg_coarsen");
    k_mg_coarsen<TF, TC><<<stream_blocks((long long)cnx * cny * cnz), LIN_BLOCK, 0, st>>>(
        A, cnx, cny, cnz, dc, wc[0], wc[1], wc[2], wpc ? wpc[0] : nullptr,
        wpc ? wpc[1] : nullptr, wpc ? wpc[2] : nullptr);
    return end();
}
template <typename T>
cudaError_t LinLaunch::diag_faces(const Op<T>& A, T* diag) {
    begin("mg_diag_faces");
    k_mg_diag_faces<T><<<stream_blocks(A.N), LIN_BLOCK, 0, st>>>(A, diag);
    return end();
}
template <typename TF, typename TO>
cudaError_t LinLaunch::level_prep(const Op<TF>& A, double omega, TO* wid, TO* loc) {
    begin("mg_level_prep");
    k_mg_level_prep<TF, TO><<<stream_blocks(A.N), LIN_BLOCK, 0, st>>>(A, omega, wid, loc);
    return end();
}
cudaError_t LinLaunch::cast_op(const Op<double>& A, float* d, float* const* w, float* const* wp) {
    begin("mg_cast_op");
    k_cast_op<<<stream_blocks(A.N), LIN_BLOCK, 0, st>>>(A, d, w[0], w[1], w[2],
                                                        wp ? wp[0] : nullptr,
                                                        wp ? wp[1] : nullptr,
                                                        wp ? wp[2] : nullptr);
    return end();
}
cudaError_t LinLaunch::to_f32(long long N, const double* a, float* b) {
    begin("mg_to_f32");
    if ((((unsigned long long)a | (unsigned long long)b) & 15ull) == 0)
        k_to_f32<true><<<stream_blocks((N + 3) / 4), LIN_BLOCK, 0, st>>>(N, a, b, skip);
    else
        k_to_f32<false><<<stream_blocks(N), LIN_BLOCK, 0, st>>>(N, a, b, skip);
    return end();
}
cudaError_t LinLaunch::from_f32_dot(long long N, const float* x, const double* r, double* z,
                                    double* part, int& nparts) {
    nparts = stream_blocks(N);
    begin("mg_from_f32_dot");
    k_from_f32_dot<<<nparts, LIN_BLOCK, 0, st>>>(N, x, r, z, part);
    return end();
}

template cudaError_t LinLaunch::smooth<double>(const Op<double>&, const double*, const double*,
                                               double*, double, int);
template cudaError_t LinLaunch::smooth<float>(const Op<float>&, const float*, const float*,
                                              float*, float, int);
template cudaError_t LinLaunch::coarse_solve<double>(const Op<double>&, const double*, double*,
                                                     double*, double, int);
template cudaError_t LinLaunch::coarse_solve<float>(const Op<float>&, const float*, float*, float*,
                                                    float, int);
template cudaError_t LinLaunch::restrict_res<double>(const Op<double>&, const double*,
                                                     const double*, int, int, int, double*);
template cudaError_t LinLaunch::restrict_res<float>(const Op<float>&, const float*, const float*,
                                                    int, int, int, float*);
template cudaError_t LinLaunch::prolong<double>(int, int, int, int, int, const double*, double*);
template cudaError_t LinLaunch::prolong<float>(int, int, int, int, int, const float*, float*);
template cudaError_t LinLaunch::coarsen<double, double>(const Op<double>&, int, int, int, double*,
                                                        double* const*, double* const*);
template cudaError_t LinLaunch::coarsen<double, float>(const Op<double>&, int, int, int, float*,
                                                       float* const*, float* const*);
template cudaError_t LinLaunch::coarsen<float, float>(const Op<float>&, int, int, int, float*,
                                                      float* const*, float* const*);
template cudaError_t LinLaunch::diag_faces<double>(const Op<double>&, double*);
template cudaError_t LinLaunch::diag_faces<float>(const Op<float>&, float*);
template cudaError_t LinLaunch::level_prep<double, double>(const Op<double>&, double, double*,
                                                           double*);
template cudaError_t LinLaunch::level_prep<double, float>(const Op<double>&, double, float*, float*);
template cudaError_t LinLaunch::level_prep<float, float>(const Op<float>&, double, float*, float*);

}  // namespace rhi
