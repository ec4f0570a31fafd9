// Learned rank seed of ADC2 (internal interface; see tdeig.h for the model).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tdeig.h"

#define MLP_IN TDEIG_MLP_IN
#define MLP_H TDEIG_MLP_HIDDEN
#define MLP_P TDEIG_MLP_PARAMS
#define MLP_OFF_B1 (MLP_H * MLP_IN)
#define MLP_OFF_W2 (MLP_OFF_B1 + MLP_H)
#define MLP_OFF_B2 (MLP_OFF_W2 + MLP_H * MLP_H)
#define MLP_OFF_W3 (MLP_OFF_B2 + MLP_H)
#define MLP_OFF_B3 (MLP_OFF_W3 + MLP_H)

// Features of one HSS node: rows [s0, s1) of a merge with K survivors out of n.
struct NodeFeatDesc {
    const double *d, *gam, *mu, *uh;
    int K, n, s0, s1;
    float* out;   // MLP_IN floats
};

void mlp_launch_features(const NodeFeatDesc* dev, int count, cudaStream_t st);
// y = model(X) (perm: optional row indices into X/t, n rows); with grad != NULL
// also accumulates the gradient of 0.5 sum_i (y_i - t_i)^2 / n_total into grad
// and, when loss != NULL, the loss into *loss (both zeroed by the caller).
void mlp_launch(const float* params, const float* mean, const float* stdv, const float* X,
                const float* t, const int* perm, int n, int n_total, float* y, float* grad,
                float* loss, cudaStream_t st);
// One Adam step; clears grad.
void mlp_launch_adam(float* params, float* grad, float* m, float* v, float lr, int step,
                     cudaStream_t st);
