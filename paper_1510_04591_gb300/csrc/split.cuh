// Split-precision products on the tensor cores (internal interface).
//
// C = alpha op(A) op(B) + beta C for FP64 operands, computed from 16-bit
// slices: every row i of op(A) is scaled by 2^-e_i (e_i its exponent bound)
// and cut into s signed beta-bit integer digits t_p, stored as t_p 2^(-beta p)
// (exact in BF16 for beta <= 8, in FP16 for beta <= 11; the 7-bit form uses
// balanced digits, |t_p| <= 64 below the top one), so that
//   op(A)[i, k] ~= 2^(e_i - beta) sum_p S_p[i, k]
// (likewise the columns of op(B) with 2^f_j).  A slice-pair product S_p S_q^T
// is an integer sum scaled by 2^(-beta (p + q)); pairs with p + q <= s - 1
// are accumulated on the tensor cores in FP32, one accumulator per level
// p + q (exact while the level's integer sum stays below 2^24, which bounds
// the k-range, `chunk`, summed before a drain), drained into a double-float
// (FP32 hi + lo) sum, converted to
// FP64 and scaled by 2^(e_i + f_j - 2 beta).  Dropped pairs and truncated
// digits bound the error by about 2^(e_i + f_j) K 2^(-beta s) per entry.
// Kinds: SPLIT_OZAKI (beta 7, s = ceil(bits / 7)), SPLIT_BF16X2 (beta 8, s 2:
// a hi + lo pair), SPLIT_FP16X2 (FP16 slices, beta 11, s 2; its FP32
// accumulation is not exact).
#pragma once

#include <cuda_bf16.h>

#include <vector>

#include "hss.cuh"

// element (r, k) of the operand being sliced: X[r*sr + col(k)*sk], col(k) = gk ? gk[k] : k,
// for k < K1; X2[r*sr2 + (k - K1)*sk2] for K1 <= k < K (a second term along k)
struct SliceDesc {
    const double* X;
    const int* gk;
    long long sr, sk;
    const double* X2;
    long long sr2, sk2;
    int K1;
    int rows, K, Kp, s, beta;
    const int* mask;    // optional: entry (r, k) is zero when mask[r] == mask[k]
    int f16;            // slices are FP16 (else BF16)
    __nv_bfloat16* S;   // slice p, row r at S + (p * rows + r) * Kp (16-bit values)
    int* e;             // exponent bound per row: max |row| < 2^e
    int t_exp, t_sl;    // first tile of this operand in the exponent and slicing launches
    int t_fu;           // first tile in the one-pass launch (operands with short rows)
    // optional: rows (when dyn_rows) and K read from *dynK at run time; rows, K are
    // then upper bounds (see GemmDesc::dynK)
    const int* dynK;
    int dyn_rows;
    // optional: the exponent bounds of the transposed twin operand (same X and
    // mask, rows and k swapped: ADC2's Z = Qhat^T Omega beside Y = Qhat Omega),
    // raised from this operand's exponent pass, which has every entry in hand;
    // the twin then has no exponent tiles of its own
    int* twin_e;
};

// One slice-pair product C = alpha 2^(ea+eb) sum_{p+q<=s-1} ... + betac C.
struct SplitGemmDesc {
    const __nv_bfloat16* SA;   // s slices of op(A), M x Kp each
    const __nv_bfloat16* SB;   // s slices of op(B)^T, N x Kp each
    const int* ea;
    const int* eb;
    int M, N, Kp, s, beta;
    double* C;
    int ldc;
    const int* ccol;
    double alpha, betac;
    int rsplit, ktop_end, kbot_beg;   // block-structured update: k ranges of the row halves
    int chunk, f16;                   // k-range summed exactly before a drain; FP16 slices
    int tile0, tiles_m;
    // TMA tensor maps (device CUtensorMap) of the slices: dims (Kp, rows, s),
    // box (32, 128 | 32, s), 64-byte swizzle
    const void *tmA, *tmB;
    int tiles_n;                      // column tiles (of the upper bound N with dynK)
    const int* dynK;                  // optional device sizes (see GemmDesc::dynK)
    const int* dynG;
};

// Tensor-core (tcgen05) slice-pair products: tile 128 x 32 per CTA, one TMEM
// accumulator per level p + q (at most 8).
#define UM_BM 128
#define UM_BN 32
#define UM_BK 32

enum { SPLIT_OZAKI = 0, SPLIT_BF16X2 = 1, SPLIT_FP16X2 = 2 };
struct SplitPrec {
    int beta, s, chunk, f16, nacc;
};
SplitPrec split_prec(int kind, int bits);
// Persistent tcgen05 launch over `tiles` output tiles of ng problems; tile0[i]
// (device) is the first tile of problem i; nacc: TMEM accumulators, one per
// level p + q (s of them).
void umma_launch(const SplitGemmDesc* dev, const int* tile0, int ng, int tiles, int smax, int nacc,
                 int* status, cudaStream_t st);
size_t umma_smem_bytes(int smax, int ng, int* nstages);

struct SplitWS {
    char* base = nullptr;
    size_t cap = 0;
};

// Significant bits the slices keep (beta * s >= this): products feeding the
// eigenvectors, and the sampling products of ADC2 (Phi = Y - D Omega cancels).
#define TD_SPLIT_BITS 40
#define TD_SAMPLE_BITS 56

// status: device word that receives TD_STATUS_TIMEOUT when a bounded wait expires.
double split_launch_gemm(const std::vector<GemmDesc>& g, SplitWS& ws, cudaStream_t st, int* rc,
                         int* status, int kind, int bits);

// A split-product launch prepared ahead of its kernels (descriptors, tensor maps
// and tile offsets already in device memory): prepared before a CUDA-graph
// capture, run inside it.
struct SplitLaunch {
    SliceDesc* dsl = nullptr;
    int nop = 0;
    long long nexp = 0, nsl = 0, nfu = 0;
    SplitGemmDesc* dsg = nullptr;
    int* dt0 = nullptr;
    int ng = 0, tiles = 0;
    int* ebase = nullptr;
    size_t erows = 0;
    SplitPrec pr{};
    double flops = 0, tflops = 0, sbytes = 0, ebytes = 0, fbytes = 0;
    char note[160] = {0};
};
// Bytes of the slices of a launch (returned) and of its descriptors (*desc_bytes).
size_t split_launch_bytes(const std::vector<GemmDesc>& g, int kind, int bits, size_t* desc_bytes);
// Grows the split workspace to at least `bytes` (synchronising st first).
int split_reserve(SplitWS& ws, size_t bytes, cudaStream_t st);
// Descriptors at desc, slices at slices (both in device memory, 256-aligned).
int split_prepare_at(const std::vector<GemmDesc>& g, char* desc, char* slices, cudaStream_t st,
                     int kind, int bits, SplitLaunch* L);
void split_run(const SplitLaunch& L, int* status, cudaStream_t st, int* rc);
// Work counters of the launches go to td_ctx() (common.cuh).
void split_free(SplitWS& ws);
