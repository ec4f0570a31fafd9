// HSS update path (Algorithms 2 and 3, SRRSC) -- internal interface.
#pragma once

#include <functional>
#include <string>
#include <vector>

#include "../../include/tdeig.h"
#include "common.cuh"

// Growable device arena owned by the handle for the HSS generators and the
// Algorithm 3 intermediates.
struct HssWS {
    char* base = nullptr;
    size_t cap = 0;
};

// C[M x N] = alpha op(A)[M x Kd] op(B)[Kd x N] + beta C, column-major.
//   op(A)[i, k] = transA ? A[k + i lda] : A[i + col(k) lda], col(k) = acol ? acol[k] : k
//   op(B)[k, j] = transB ? B[j + k ldb] : B[k + j ldb]
//   C column j is written to column ccol ? ccol[j] : j
struct GemmDesc {
    const double* A;
    const double* B;
    double* C;
    const int* acol;
    const int* ccol;
    int M, N, Kd, lda, ldb, ldc;
    int transA, transB;
    double alpha, beta;
    int tile0, tiles_m;
    // optional block structure (split products only): rows < rsplit use k < ktop_end,
    // rows >= rsplit use k >= kbot_beg (the other entries of op(A) are zero); 0 = none
    int rsplit, ktop_end, kbot_beg;
    // optional (split products only): entry (r, k) of op(A) is taken as zero when
    // amask[r] == amask[k] (ADC2 sampling of the off-diagonal part of Qhat)
    const int* amask;
    // optional (split products only): a second term along k, C = alpha (op(A) op(B) +
    // op(A2) op(B2)) + beta C, op(A2) M x Kd2, op(B2) Kd2 x N (no column gather);
    // Kd2 = 0: none
    const double* A2;
    const double* B2;
    int Kd2, lda2, ldb2, transA2, transB2;
    // optional (split products only): sizes known only on the device, so that the
    // launch sequence needs no host read-back (CUDA-graph capture).  N and Kd
    // above are then upper bounds; the actual N = Kd = *dynK, and with the block
    // structure ktop_end = dynG[0] + dynG[1], kbot_beg = dynG[0].
    const int* dynK;
    const int* dynG;
};

// out[a + b ld] = uhat[row] v[col] / (d[row] - lambda[col]) (Remark 1), for
// row = rows ? rows[a] : r0 + a and col = cols ? cols[b] : c0 + b.
struct FillDesc {
    double* out;
    int ld, nr, nc;
    const int* rows;
    int r0;
    const int* cols;
    int c0;
    const double *d, *gam, *mu, *uhat, *v;
    int tile0, tiles_r;
};

// Row interpolative decomposition Phi ~= U Phi[piv, :] (m x s input).
struct IdDesc {
    const double* Phi;
    int ldphi, m, s;
    // global index of local row a: rowmap ? (a < n1 ? rowmap[a] : rowmap2[a - n1]) : rowbase + a
    const int* rowmap;
    const int* rowmap2;
    int n1;
    int rowbase;
    double* U;          // m x rank, leading dimension ldu
    int ldu;
    int* out_idx;       // global indices of the skeleton rows
    int* out_piv;       // local skeleton rows
    int* out_rank;
};

// dst[a + c ldd] = src[piv[a] + c lds], a < nr, c < ncols.
struct GatherDesc {
    const double* src;
    int lds;
    const int* piv;
    int nr;
    double* dst;
    int ldd, ncols;
};

// One HSS block row (side 0: rows = node rows, entries uhat_r v_c / (d_r - lambda_c))
// or block column (side 1: rows = node columns, entries v_r uhat_c / (d_c - lambda_r))
// against every index outside the node's span [s0, s1), compressed by complete-pivoting
// elimination on its Cauchy generators (ADC1).
struct SrrscDesc {
    int m;                 // rows: global index of row a = a < n1 ? map1[a] : (map2 ? map2[a - n1] : base + a)
    const int* map1;
    int n1;
    const int* map2;
    int base;
    int s0, s1, K, side, kcap;
    const double *d, *gam, *mu, *uh, *v;   // Cauchy generators of the merge
    float* invd;           // ncols x 8: each column's pole data for the pivot search
    double *g, *h;         // generators, m and ncols
    float *gf, *hf;        // FP32 copies for the pivot search
    unsigned char *actr, *actc;
    double* mult;          // m x kcap elimination multipliers
    double* U;             // m x rank interpolation matrix, leading dimension ldu
    int ldu;
    int *out_idx, *out_piv, *out_rank;
};

struct RankDesc {
    const double *d, *gam;
    int K, nl;
    int* bounds;  // nl + 1 entries, in/out
    int* r_out;
};

// Stage launchers (the stage entry points of include/tdeig.h).
void hss_launch_rank_estimate(const RankDesc* dev, int nr, double eps, int cap, int shift,
                              cudaStream_t st);
// TDEIG_EINVAL when an m x s ID does not fit the kernel's shared memory.
int hss_launch_id(const IdDesc* dev, int nd, int smax, int mmax, double tol, cudaStream_t st);
void hss_launch_philox_words(const unsigned* ctr, const unsigned* key, unsigned* out, int64_t n,
                             cudaStream_t st);
void hss_launch_gaussian(double* Om, int K, int s, unsigned long long seed, unsigned stream,
                         cudaStream_t st);

// Launches one grouped product; returns its algorithmic flops (2 M N Kd summed).
double hss_launch_gemm(const std::vector<GemmDesc>& g, GemmDesc* dev, cudaStream_t st);
void hss_free(HssWS& w);
// mark(name) records a timing event that starts sub-stage `name` (sampling,
// construction, multiplication) on the solve's stream.  With split != NULL the
// sampling and Algorithm 3 products run as split-precision tensor-core products.
struct SplitWS;
// Learned rank seed of ADC2 (TDEIG_FLAG_MLP_SEED / TDEIG_FLAG_RECORD).
struct HssLearn {
    const float* model = nullptr;        // device: params | mean | std (seed only)
    bool seed = false, record = false;
    std::vector<float>* records = nullptr;   // 8 floats per recorded node
    int fallbacks = 0;                   // merges rebuilt with the estimate
};
int hss_update_level(const tdeig_options& opt, int variant, int prec,
                     const std::vector<MergeDesc>& merges, const MergeDesc* dev_merges,
                     const std::vector<int>& K, const LevelWS& lws, HssWS& hws, int* status,
                     cudaStream_t st, std::string& stats,
                     const std::function<int(const char*)>& mark, SplitWS* split,
                     HssLearn* learn);
