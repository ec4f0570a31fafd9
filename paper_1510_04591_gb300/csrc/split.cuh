// Split-precision products on the tensor cores (internal interface).
//
// C = alpha op(A) op(B) + beta C for FP64 operands, computed from BF16 slices:
// every row i of op(A) is scaled by 2^-e_i (e_i the exponent bound of the row)
// and cut into s signed beta-bit integer digits t_p (|t_p| < 2^beta), so that
//   op(A)[i, k] ~= 2^e_i sum_p t_p[i, k] 2^(-beta (p+1))
// (likewise the columns of op(B) with 2^f_j).  beta is the largest value with
// (2^beta - 1)^2 K <= 2^24, so each slice-pair product sum_k t_p t_q is an
// integer that FP32 accumulation on the tensor cores represents exactly.  Pairs
// with p + q <= s - 1 are accumulated per output entry in a double-float (FP32
// hi + lo) sum, converted to FP64 and scaled by 2^(e_i + f_j) at the end.
// Dropped pairs and truncated digits bound the error by about
// 2^(e_i + f_j) K 2^(-beta s) per entry.
#pragma once

#include <vector>

#include "hss.cuh"

struct SplitWS {
    char* base = nullptr;
    size_t cap = 0;
};

// Number of significant bits the slices keep (beta * s >= this).
#define TD_SPLIT_BITS 40

double split_launch_gemm(const std::vector<GemmDesc>& g, SplitWS& ws, cudaStream_t st, int* rc);
// Tensor-core work issued by split products so far: 2 M N K per slice pair.
extern double g_split_tensor_flops;
void split_free(SplitWS& ws);
// beta and s used for a contraction of length K.
void split_params(int K, int* beta, int* s);
