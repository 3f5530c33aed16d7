// Learned Newton initial guess (an addition to the paper's method, whose Sec. 3.2 leaves the
// initial iterate free and whose Sec. 3.2.4 uses an explicit predictor): a per-cell MLP
// 13 -> 64 -> 64 -> 64 -> 6 with SiLU that predicts the state at t^{n+1} from the state at
// t^n and the change of the previous step.
//
//   features  log10 E/u_E, log10 e/u_e, log10 x_HI, log10 x_HeI, log10 x_HeII, log10 n_H/u_n,
//             log10(dt Gamma_HI + 1e-30), log10(1 + 4 pi eta dt / E), log10(dt / 1e12 s),
//             log10 E/E^{n-1}, log10 e/e^{n-1}, logit x_HI - logit x_HI^{n-1},
//             log10(dt / dt^{n-1}) (the last four 0 before a first step)
//   outputs   log10 E'/E, log10 e'/e, logit x_HI', He fraction logits (softmax)
//
// Inference runs on the tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulation)
// with the layer activations chained in registers; training runs FP32 on the CUDA cores with
// one thread per sample, a deterministic weight-gradient reduction and Adam.
#include <cmath>

#include "rhi_mlp.cuh"

namespace rhi {

namespace {

constexpr int INF_WARPS = 4;                  // warps per inference block
constexpr int TRAIN_BLOCK = 128;

// ------------------------------------------------------------------------------------------
// features of one cell (FP32 from the FP64 state)

__device__ __forceinline__ float log10_clamped(double x) {
    // FP32 logarithm of a positive ratio formed in FP64, clamped into the FP32 range
    return log10f(fminf(fmaxf((float)x, 1e-37f), 1e37f));
}

__device__ __forceinline__ void cell_features(const MlpArgs& A, long long c, float (&f)[MLP_IN]) {
    // ratios in FP64 (the source ratio and the field leave the FP32 range in cells the
    // radiation has not reached), logarithms in FP32
    const double E = A.E[c], e = A.e[c], nH = A.nH[c];
    const double inH = 1.0 / nH;
    f[0] = log10_clamped(E * A.iu_E);
    f[1] = log10_clamped(e * A.iu_e);
    f[2] = log10_clamped(fmax(A.n[c] * inH, 1e-30));
    if (A.ns == 3) {
        const double inHe = inH / A.y_he;
        f[3] = log10_clamped(fmax(A.n[A.N + c] * inHe, 1e-30));
        f[4] = log10_clamped(fmax(A.n[2 * A.N + c] * inHe, 1e-30));
    } else {
        f[3] = 0.0f;
        f[4] = 0.0f;
    }
    f[5] = log10_clamped(nH * A.iu_n);
    f[6] = log10_clamped(A.dt * A.gam_per_E * E + 1e-30);
    f[7] = log10f(1.0f + fminf((float)(A.src[c] * A.dt / E), 1e37f));
    f[8] = log10_clamped(A.dt * 1e-12);
    if (A.E_p) {
        // the previous step's change: ratios in FP64, the logit difference in FP64 (neutral
        // cells sit within 1e-16 of x_HI = 1), rounded to FP32
        f[9] = log10_clamped(E / A.E_p[c]);
        f[10] = log10_clamped(e / A.e_p[c]);
        const double x1 = fmin(fmax(A.n[c] * inH, 1e-30), 1.0 - 1e-16);
        const double x0 = fmin(fmax(A.n_p[c] * inH, 1e-30), 1.0 - 1e-16);
        f[11] = (float)((log(x1) - log1p(-x1)) - (log(x0) - log1p(-x0)));
        f[12] = A.ldt_ratio;
    } else {
        f[9] = f[10] = f[11] = f[12] = 0.0f;
    }
}

__global__ void k_mlp_features(const MlpArgs A, float* __restrict__ X) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= A.N) return;
    float f[MLP_IN];
    cell_features(A, c, f);
#pragma unroll
    for (int q = 0; q < MLP_IN; ++q) X[c * MLP_IN + q] = f[q];
}

// targets of the step (E0, e0, n0) -> (E, e, n) of MlpArgs
__global__ void k_mlp_targets(const MlpArgs A, const double* __restrict__ E0,
                              const double* __restrict__ e0, const double* __restrict__ n0,
                              float* __restrict__ Y) {
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= A.N) return;
    float* y = Y + c * MLP_OUT;
    y[0] = (float)log10(A.E[c] / E0[c]);
    y[1] = (float)log10(A.e[c] / e0[c]);
    const double nH = A.nH[c];
    const double x = fmin(fmax(A.n[c] / nH, 1e-30), 1.0 - 1e-16);
    y[2] = (float)(log(x) - log1p(-x));
    if (A.ns == 3) {
        const double nHe = A.y_he * nH;
        const double f0 = A.n[A.N + c] / nHe, f1 = A.n[2 * A.N + c] / nHe;
        const double l0 = log(fmax(f0, 1e-30)), l1 = log(fmax(f1, 1e-30));
        const double l2 = log(fmax(1.0 - f0 - f1, 1e-30));
        const double m = (l0 + l1 + l2) / 3.0;
        y[3] = (float)(l0 - m);
        y[4] = (float)(l1 - m);
        y[5] = (float)(l2 - m);
    } else {
        y[3] = y[4] = y[5] = 0.0f;
    }
}

// ------------------------------------------------------------------------------------------
// tensor-core inference

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ float silu_f(float z) { return z / (1.0f + __expf(-z)); }

// one hidden layer on a 16-row tile: in = A fragments over KS k-steps, out = 8 n-tiles
template <int KS, int RS>
__device__ __forceinline__ void hidden_layer(const uint32_t (&a)[4][4], const __nv_bfloat16* W,
                                             const float* b, float (&acc)[8][4], int g, int t) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float b0 = b[8 * j + 2 * t], b1 = b[8 * j + 2 * t + 1];
        acc[j][0] = b0; acc[j][1] = b1; acc[j][2] = b0; acc[j][3] = b1;
#pragma unroll
        for (int s = 0; s < KS; ++s) {
            const __nv_bfloat16* w = W + (8 * j + g) * RS + 16 * s + 2 * t;
            mma_bf16(acc[j], a[s], *reinterpret_cast<const uint32_t*>(w),
                     *reinterpret_cast<const uint32_t*>(w + 8));
        }
    }
}

// SiLU of 8 n-tiles into the A fragments of the next layer's 4 k-steps
__device__ __forceinline__ void to_fragments(const float (&acc)[8][4], uint32_t (&a)[4][4]) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        a[s][0] = pack_bf16(silu_f(acc[2 * s][0]), silu_f(acc[2 * s][1]));
        a[s][1] = pack_bf16(silu_f(acc[2 * s][2]), silu_f(acc[2 * s][3]));
        a[s][2] = pack_bf16(silu_f(acc[2 * s + 1][0]), silu_f(acc[2 * s + 1][1]));
        a[s][3] = pack_bf16(silu_f(acc[2 * s + 1][2]), silu_f(acc[2 * s + 1][3]));
    }
}

// MODE 0: outputs for given features X (n rows) into Y;  MODE 1: guess for every cell of the
// state (features computed here), decoded into the work iterate (e_c, n, E) and its opacity
template <int MODE>
__global__ void __launch_bounds__(32 * INF_WARPS) k_mlp_infer(const MlpArgs A,
                                                              const MlpPacked* __restrict__ pk,
                                                              const float* __restrict__ X,
                                                              float* __restrict__ Y,
                                                              long long n_rows) {
    __shared__ MlpPacked sw;
    __shared__ __nv_bfloat16 xs[INF_WARPS][32][24];
    __shared__ float os[INF_WARPS][32][8];
    // stage the packed weights
    {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(pk);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&sw);
        for (int q = threadIdx.x; q < (int)(sizeof(MlpPacked) / 4); q += blockDim.x) dst[q] = src[q];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const long long rows = (MODE == 0) ? n_rows : A.N;
    const long long ntiles = (rows + 31) / 32;
    for (long long tile = blockIdx.x * (long long)INF_WARPS + warp; tile < ntiles;
         tile += (long long)gridDim.x * INF_WARPS) {
        const long long c = tile * 32 + lane;
        float f[MLP_IN];
        if (c < rows) {
            if (MODE == 0) {
#pragma unroll
                for (int q = 0; q < MLP_IN; ++q) f[q] = X[c * MLP_IN + q];
            } else {
                cell_features(A, c, f);
            }
        } else {
#pragma unroll
            for (int q = 0; q < MLP_IN; ++q) f[q] = sw.mean[q];
        }
        bool ood = false;
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const float xn = q < MLP_IN ? (f[q] - sw.mean[q]) * sw.iscale[q] : 0.0f;
            ood |= A.ood > 0.0f && fabsf(xn) > A.ood;
            xs[warp][lane][q] = __float2bfloat16_rn(xn);
        }
        __syncwarp();
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int r0 = 16 * half + g;
            uint32_t a[4][4];
            a[0][0] = *reinterpret_cast<const uint32_t*>(&xs[warp][r0][2 * t]);
            a[0][1] = *reinterpret_cast<const uint32_t*>(&xs[warp][r0 + 8][2 * t]);
            a[0][2] = *reinterpret_cast<const uint32_t*>(&xs[warp][r0][2 * t + 8]);
            a[0][3] = *reinterpret_cast<const uint32_t*>(&xs[warp][r0 + 8][2 * t + 8]);
            float acc[8][4];
            hidden_layer<1, RS1>(a, sw.W1, sw.b1, acc, g, t);
            to_fragments(acc, a);
            hidden_layer<4, RS2>(a, sw.W2, sw.b2, acc, g, t);
            to_fragments(acc, a);
            hidden_layer<4, RS2>(a, sw.W3, sw.b3, acc, g, t);
            to_fragments(acc, a);
            float o[4] = {sw.b4[2 * t], sw.b4[2 * t + 1], sw.b4[2 * t], sw.b4[2 * t + 1]};
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                const __nv_bfloat16* w = sw.W4 + g * RS2 + 16 * s + 2 * t;
                mma_bf16(o, a[s], *reinterpret_cast<const uint32_t*>(w),
                         *reinterpret_cast<const uint32_t*>(w + 8));
            }
            os[warp][r0][2 * t] = o[0];
            os[warp][r0][2 * t + 1] = o[1];
            os[warp][r0 + 8][2 * t] = o[2];
            os[warp][r0 + 8][2 * t + 1] = o[3];
        }
        __syncwarp();
        if (c < rows) {
            const float* o = os[warp][lane];
            if (MODE == 0) {
#pragma unroll
                for (int q = 0; q < MLP_OUT; ++q) Y[c * MLP_OUT + q] = o[q];
            } else {
                // decode (FP32 transcendentals; the logit of the old fraction in FP64, where
                // neutral cells sit within 1e-16 of 1); cells whose predicted change stays
                // below the gate, or whose inputs left the training range, keep U^n
                const double E0 = A.E[c], e0 = A.e[c], nH = A.nH[c];
                const double x0 = fmin(fmax(A.n[c] / nH, 1e-30), 1.0 - 1e-16);
                float change = fmaxf(fabsf(o[0]), fabsf(o[1]));
                change = fmaxf(change, fabsf(o[2] - (float)(log(x0) - log1p(-x0))));
                const double xHI = 1.0 / (1.0 + (double)expf(-o[2]));
                double nHeI = 0.0, nHeII = 0.0;
                if (A.ns == 3) {
                    // softmax normalised in FP64: n_HeI + n_HeII stays below n_He to rounding,
                    // so the derived n_HeIII of the guess is not negative beyond the positivity
                    // cap's tolerance (an FP32 sum can overshoot by 1e-7 n_He and freeze the cell)
                    const double nHe = A.y_he * nH;
                    const float mx = fmaxf(o[3], fmaxf(o[4], o[5]));
                    const double z0 = expf(o[3] - mx), z1 = expf(o[4] - mx), z2 = expf(o[5] - mx);
                    const double iz = 1.0 / (z0 + z1 + z2);
                    const double f0 = A.n[A.N + c] / nHe, f1 = A.n[2 * A.N + c] / nHe;
                    const double f2 = 1.0 - f0 - f1;
                    change = fmaxf(change, fabsf(logf((float)fmax(z0 * iz, 1e-30)) - logf((float)fmax(f0, 1e-30))));
                    change = fmaxf(change, fabsf(logf((float)fmax(z1 * iz, 1e-30)) - logf((float)fmax(f1, 1e-30))));
                    change = fmaxf(change, fabsf(logf((float)fmax(z2 * iz, 1e-30)) - logf((float)fmax(f2, 1e-30))));
                    nHeI = nHe * (z0 * iz);
                    nHeII = nHe * (z1 * iz);
                }
                const long long N = A.N;
                double* U = A.U0;
                if (change < A.gate || ood) {
                    U[c] = 0.0;
                    for (int s = 0; s < A.ns; ++s) U[(1 + s) * N + c] = A.n[s * N + c];
                    U[(1 + A.ns) * N + c] = E0;
                } else {
                    U[c] = A.isothermal ? 0.0 : e0 * (double)expm1f(2.302585093f * o[1]);
                    U[N + c] = nH * xHI;
                    if (A.ns == 3) {
                        U[2 * N + c] = nHeI;
                        U[3 * N + c] = nHeII;
                    }
                    U[(1 + A.ns) * N + c] = E0 * (double)exp10f(o[0]);
                }
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------------------------------
// FP32 training: one thread per sample

struct TrainW {
    float W1[MLP_HID * MLP_IN], b1[MLP_HID];
    float W2[MLP_HID * MLP_HID], b2[MLP_HID];
    float W3[MLP_HID * MLP_HID], b3[MLP_HID];
    float W4[MLP_OUT * MLP_HID], b4[MLP_OUT];
    float mean[MLP_IN], scale[MLP_IN];
};
static_assert(sizeof(TrainW) == RHI_MLP_NWEIGHTS * sizeof(float), "weight layout");

__device__ __forceinline__ float sig_f(float z) { return 1.0f / (1.0f + expf(-z)); }

// forward + backward of one sample: stores the per-sample deltas d1, d2, d3 (64 each), g4 (6)
// and the activations h0 (9), h1, h2, h3 (64 each) for the weight-gradient reduction, and the
// squared error into the block partials
__global__ void __launch_bounds__(TRAIN_BLOCK) k_mlp_fwd_bwd(const float* __restrict__ w,
                                                             const float* __restrict__ X,
                                                             const float* __restrict__ Y,
                                                             long long m, float inv_norm,
                                                             float* __restrict__ act,
                                                             float* __restrict__ del,
                                                             double* __restrict__ partials) {
    extern __shared__ float smem[];
    TrainW& W = *reinterpret_cast<TrainW*>(smem);
    for (int q = threadIdx.x; q < RHI_MLP_NWEIGHTS; q += blockDim.x) smem[q] = w[q];
    __syncthreads();
    const long long s = blockIdx.x * (long long)TRAIN_BLOCK + threadIdx.x;
    double se = 0.0;
    if (s < m) {
        float h0[MLP_IN], z1[MLP_HID], z2[MLP_HID], z3[MLP_HID], h[MLP_HID], out[MLP_OUT];
        for (int k = 0; k < MLP_IN; ++k) h0[k] = (X[s * MLP_IN + k] - W.mean[k]) / W.scale[k];
        for (int n = 0; n < MLP_HID; ++n) {
            float a = W.b1[n];
            for (int k = 0; k < MLP_IN; ++k) a += W.W1[n * MLP_IN + k] * h0[k];
            z1[n] = a;
        }
        for (int k = 0; k < MLP_HID; ++k) h[k] = z1[k] * sig_f(z1[k]);
        for (int n = 0; n < MLP_HID; ++n) {
            float a = W.b2[n];
            for (int k = 0; k < MLP_HID; ++k) a += W.W2[n * MLP_HID + k] * h[k];
            z2[n] = a;
        }
        for (int k = 0; k < MLP_HID; ++k) h[k] = z2[k] * sig_f(z2[k]);
        for (int n = 0; n < MLP_HID; ++n) {
            float a = W.b3[n];
            for (int k = 0; k < MLP_HID; ++k) a += W.W3[n * MLP_HID + k] * h[k];
            z3[n] = a;
        }
        for (int k = 0; k < MLP_HID; ++k) h[k] = z3[k] * sig_f(z3[k]);
        float g4[MLP_OUT];
        for (int n = 0; n < MLP_OUT; ++n) {
            float a = W.b4[n];
            for (int k = 0; k < MLP_HID; ++k) a += W.W4[n * MLP_HID + k] * h[k];
            out[n] = a;
            const float d = a - Y[s * MLP_OUT + n];
            se += (double)d * d;
            g4[n] = 2.0f * d * inv_norm;
        }
        // activations for the weight gradients: h0 | h1 | h2 | h3
        float* as = act + s * ACT_STRIDE;
        for (int k = 0; k < MLP_IN; ++k) as[k] = h0[k];
        for (int k = 0; k < MLP_HID; ++k) {
            as[MLP_IN + k] = z1[k] * sig_f(z1[k]);
            as[MLP_IN + MLP_HID + k] = z2[k] * sig_f(z2[k]);
            as[MLP_IN + 2 * MLP_HID + k] = h[k];
        }
        // deltas: d1 | d2 | d3 | g4
        float* ds = del + s * DEL_STRIDE;
        for (int n = 0; n < MLP_OUT; ++n) ds[3 * MLP_HID + n] = g4[n];
        float d3[MLP_HID];
        for (int k = 0; k < MLP_HID; ++k) {
            float a = 0.0f;
            for (int n = 0; n < MLP_OUT; ++n) a += W.W4[n * MLP_HID + k] * g4[n];
            const float sg = sig_f(z3[k]);
            d3[k] = a * sg * (1.0f + z3[k] * (1.0f - sg));
            ds[2 * MLP_HID + k] = d3[k];
        }
        float d2[MLP_HID];
        for (int k = 0; k < MLP_HID; ++k) {
            float a = 0.0f;
            for (int n = 0; n < MLP_HID; ++n) a += W.W3[n * MLP_HID + k] * d3[n];
            const float sg = sig_f(z2[k]);
            d2[k] = a * sg * (1.0f + z2[k] * (1.0f - sg));
            ds[MLP_HID + k] = d2[k];
        }
        for (int k = 0; k < MLP_HID; ++k) {
            float a = 0.0f;
            for (int n = 0; n < MLP_HID; ++n) a += W.W2[n * MLP_HID + k] * d2[n];
            const float sg = sig_f(z1[k]);
            ds[k] = a * sg * (1.0f + z1[k] * (1.0f - sg));
        }
    }
    const double bs = block_sum<TRAIN_BLOCK>(se);
    if (threadIdx.x == 0) partials[blockIdx.x] = bs;
}

// weight gradients: one block per weight row (layer, n); thread k sums delta_n h_k over the
// samples in a fixed order (deterministic); the last thread of a row also sums the bias
__global__ void __launch_bounds__(MLP_HID) k_mlp_wgrad(const float* __restrict__ act,
                                                       const float* __restrict__ del, long long m,
                                                       float* __restrict__ grad) {
    // rows: layer 1: 64 rows x 9 inputs, layer 2, 3: 64 x 64, layer 4: 6 x 64
    int row = blockIdx.x, layer, n;
    if (row < MLP_HID) { layer = 0; n = row; }
    else if (row < 2 * MLP_HID) { layer = 1; n = row - MLP_HID; }
    else if (row < 3 * MLP_HID) { layer = 2; n = row - 2 * MLP_HID; }
    else { layer = 3; n = row - 3 * MLP_HID; }
    const int K = layer == 0 ? MLP_IN : MLP_HID;
    const int aoff = layer == 0 ? 0 : MLP_IN + (layer - 1) * MLP_HID;
    const int doff = layer == 3 ? 3 * MLP_HID + n : layer * MLP_HID + n;
    const int k = threadIdx.x;
    float acc = 0.0f, bacc = 0.0f;
    for (long long s = 0; s < m; ++s) {
        const float d = del[s * DEL_STRIDE + doff];
        if (k < K) acc += d * act[s * ACT_STRIDE + aoff + k];
        bacc += d;
    }
    // weight vector offsets
    const int wofs[4] = {0, MLP_HID * MLP_IN + MLP_HID,
                         MLP_HID * MLP_IN + MLP_HID + MLP_HID * MLP_HID + MLP_HID,
                         MLP_HID * MLP_IN + MLP_HID + 2 * (MLP_HID * MLP_HID + MLP_HID)};
    const int nrows = layer == 3 ? MLP_OUT : MLP_HID;
    if (k < K) grad[wofs[layer] + n * K + k] = acc;
    if (k == 0) grad[wofs[layer] + nrows * K + n] = bacc;
}

__global__ void k_mlp_adam(float* __restrict__ w, const float* __restrict__ g,
                           float* __restrict__ m1, float* __restrict__ m2, int n, float lr,
                           float b1t, float b2t) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const float b1 = 0.9f, b2 = 0.999f;
    const float gv = g[q];
    const float a = b1 * m1[q] + (1.0f - b1) * gv;
    const float b = b2 * m2[q] + (1.0f - b2) * gv * gv;
    m1[q] = a;
    m2[q] = b;
    w[q] -= lr * (a / (1.0f - b1t)) / (sqrtf(b / (1.0f - b2t)) + 1e-8f);
}

}  // namespace

// ------------------------------------------------------------------------------------------
// launchers

cudaError_t launch_mlp_features(const MlpArgs& A, float* X, cudaStream_t st) {
    k_mlp_features<<<(unsigned)((A.N + 255) / 256), 256, 0, st>>>(A, X);
    return cudaGetLastError();
}

cudaError_t launch_mlp_targets(const MlpArgs& A, const double* E0, const double* e0,
                               const double* n0, float* Y, cudaStream_t st) {
    k_mlp_targets<<<(unsigned)((A.N + 255) / 256), 256, 0, st>>>(A, E0, e0, n0, Y);
    return cudaGetLastError();
}

cudaError_t launch_mlp_infer(const MlpArgs& A, const MlpPacked* pk, const float* X, float* Y,
                             long long n_rows, int guess, cudaStream_t st) {
    const long long rows = guess ? A.N : n_rows;
    const long long tiles = (rows + 31) / 32;
    long long blocks = (tiles + INF_WARPS - 1) / INF_WARPS;
    if (blocks > 152LL * 8) blocks = 152LL * 8;
    if (blocks < 1) blocks = 1;
    if (guess) k_mlp_infer<1><<<(unsigned)blocks, 32 * INF_WARPS, 0, st>>>(A, pk, X, Y, n_rows);
    else k_mlp_infer<0><<<(unsigned)blocks, 32 * INF_WARPS, 0, st>>>(A, pk, X, Y, n_rows);
    return cudaGetLastError();
}

int mlp_train_block() { return TRAIN_BLOCK; }

cudaError_t launch_mlp_fwd_bwd(const float* w, const float* X, const float* Y, long long m,
                               float* act, float* del, double* partials, cudaStream_t st) {
    const unsigned blocks = (unsigned)((m + TRAIN_BLOCK - 1) / TRAIN_BLOCK);
    const size_t sm = RHI_MLP_NWEIGHTS * sizeof(float);
    cudaFuncSetAttribute(k_mlp_fwd_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_mlp_fwd_bwd<<<blocks, TRAIN_BLOCK, sm, st>>>(w, X, Y, m, 1.0f / (float)(m * MLP_OUT), act,
                                                   del, partials);
    return cudaGetLastError();
}

cudaError_t launch_mlp_wgrad(const float* act, const float* del, long long m, float* grad,
                             cudaStream_t st) {
    k_mlp_wgrad<<<3 * MLP_HID + MLP_OUT, MLP_HID, 0, st>>>(act, del, m, grad);
    return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* w, const float* g, float* m1, float* m2, int n, float lr,
                            float b1t, float b2t, cudaStream_t st) {
    k_mlp_adam<<<(n + 255) / 256, 256, 0, st>>>(w, g, m1, m2, n, lr, b1t, b2t);
    return cudaGetLastError();
}

// pack FP32 master weights into the padded BF16 inference layout
void mlp_pack(const float* w, MlpPacked* out) {
    std::memset(out, 0, sizeof(MlpPacked));
    const float* W1 = w;
    const float* b1 = W1 + MLP_HID * MLP_IN;
    const float* W2 = b1 + MLP_HID;
    const float* b2 = W2 + MLP_HID * MLP_HID;
    const float* W3 = b2 + MLP_HID;
    const float* b3 = W3 + MLP_HID * MLP_HID;
    const float* W4 = b3 + MLP_HID;
    const float* b4 = W4 + MLP_OUT * MLP_HID;
    const float* mean = b4 + MLP_OUT;
    const float* scale = mean + MLP_IN;
    for (int n = 0; n < MLP_HID; ++n) {
        for (int k = 0; k < MLP_IN; ++k) out->W1[n * RS1 + k] = __float2bfloat16(W1[n * MLP_IN + k]);
        for (int k = 0; k < MLP_HID; ++k) {
            out->W2[n * RS2 + k] = __float2bfloat16(W2[n * MLP_HID + k]);
            out->W3[n * RS2 + k] = __float2bfloat16(W3[n * MLP_HID + k]);
        }
        out->b1[n] = b1[n];
        out->b2[n] = b2[n];
        out->b3[n] = b3[n];
    }
    for (int n = 0; n < MLP_OUT; ++n) {
        for (int k = 0; k < MLP_HID; ++k) out->W4[n * RS2 + k] = __float2bfloat16(W4[n * MLP_HID + k]);
        out->b4[n] = b4[n];
    }
    for (int k = 0; k < MLP_IN; ++k) {
        out->mean[k] = mean[k];
        out->iscale[k] = 1.0f / scale[k];
    }
}

}  // namespace rhi
