// Declarations of the learned-guess MLP kernels (rhi_mlp.cu).
#pragma once

#include <cuda_bf16.h>

#include <cstring>

#include "rhi_internal.cuh"

namespace rhi {

constexpr int MLP_IN = RHI_MLP_IN, MLP_HID = RHI_MLP_HID, MLP_OUT = RHI_MLP_OUT;
constexpr int RS1 = 24;                       // padded row strides (bf16) of the packed weights
constexpr int RS2 = 72;
constexpr int ACT_STRIDE = MLP_IN + 3 * MLP_HID;     // per-sample activations h0 | h1 | h2 | h3
constexpr int DEL_STRIDE = 3 * MLP_HID + MLP_OUT;    // per-sample deltas d1 | d2 | d3 | g4

// inference weights: BF16 rows padded for conflict-free fragment loads, FP32 biases and
// the input normalisation (mean, 1 / scale)
struct MlpPacked {
    __nv_bfloat16 W1[MLP_HID * RS1];
    __nv_bfloat16 W2[MLP_HID * RS2];
    __nv_bfloat16 W3[MLP_HID * RS2];
    __nv_bfloat16 W4[8 * RS2];
    float b1[MLP_HID], b2[MLP_HID], b3[MLP_HID], b4[8];
    float mean[MLP_IN], iscale[MLP_IN];
};

struct MlpArgs {
    long long N;
    int ns;
    double y_he, iu_E, iu_e, iu_n, dt, gam_per_E;
    const double* E;
    const double* e;
    const double* n;
    const double* nH;
    const double* src;
    // the state before the last accepted step (null: none yet) and log10(dt / dt^{n-1})
    const double* E_p;
    const double* e_p;
    const double* n_p;
    float ldt_ratio;
    float gate;
    float ood;                                // |normalised feature| above this keeps U^n
    int isothermal;                           // guess keeps e_c = 0
    double* U0;                               // guess (e_c | n | E), MODE 1
};

void mlp_pack(const float* w, MlpPacked* out);
cudaError_t launch_mlp_features(const MlpArgs& A, float* X, cudaStream_t st);
cudaError_t launch_mlp_targets(const MlpArgs& A, const double* E0, const double* e0,
                               const double* n0, float* Y, cudaStream_t st);
cudaError_t launch_mlp_infer(const MlpArgs& A, const MlpPacked* pk, const float* X, float* Y,
                             long long n_rows, int guess, cudaStream_t st);
int mlp_train_block();
cudaError_t launch_mlp_fwd_bwd(const float* w, const float* X, const float* Y, long long m,
                               float* act, float* del, double* partials, cudaStream_t st);
cudaError_t launch_mlp_wgrad(const float* act, const float* del, long long m, float* grad,
                             cudaStream_t st);
cudaError_t launch_mlp_adam(float* w, const float* g, float* m1, float* m2, int n, float lr,
                            float b1t, float b2t, cudaStream_t st);

}  // namespace rhi
