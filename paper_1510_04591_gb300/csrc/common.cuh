// Internal declarations shared by the translation units of libtdeig.so.
// Not part of the public C ABI (see include/tdeig.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#define TD_EPS 1.1102230246251565e-16  // unit roundoff 2^-53
#define TD_SECULAR_MAXIT 64            // secular iteration cap per root
#define TD_STATUS_NOTCONV 1
#define TD_STATUS_LEAF 2
#define TD_STATUS_TIMEOUT 4
#define TD_STATUS_BADRANK 8
// status[TD_STATUS_SECULAR_TERMS .. +1]: 64-bit count of secular terms evaluated
// in FP64; status[TD_STATUS_SECULAR_DFTERMS .. +1]: in double-float
#define TD_STATUS_SECULAR_TERMS 2
#define TD_STATUS_SECULAR_DFTERMS 4

// One merge of the DC tree (Algorithm 1): the node covers global rows
// [g0, g0 + n); child 1 is [g0, g0 + n1), child 2 the rest.
struct MergeDesc {
    const double* qin1;    // child 1 eigenvectors, n1 x n1 column-major
    const double* qin2;    // child 2 eigenvectors, n2 x n2 column-major
    double* qout;          // this node's eigenvectors, n x n column-major
    const double* lam_in;  // children eigenvalues (child 1 then child 2), n entries
    double* lam_out;       // n entries, ascending
    double* W;             // n x n workspace: sorted, deflation-rotated diag(Q1, Q2)
    double* qhat;          // K x K workspace (capacity n x n): Cauchy-like eigenvector matrix
    const double* scale_ptr;  // the matrix scale at roots (eigenvalues are unscaled), else NULL
    const double* beta_ptr;   // scaled coupling b_k between the children (device)
    int g0, n, n1;
    int member;
    int node_id;           // node of the DC tree: root 0, children of i are 2i+1, 2i+2
    int tile0;             // first GEMM tile of this merge in the level's tile numbering
    int tiles_m;           // row tiles of this merge
    // stage entry point only (NULL in a solve): the merge vector's halves given
    // directly, z1 = last row of Q1 (n1), z2 = first row of Q2 (n2)
    const double* z1;
    const double* z2;
};

struct LeafDesc {
    double* qout;      // n x n column-major
    double* lam_out;   // n entries
    const double* scale_ptr;  // the matrix scale if the leaf is the whole matrix, else NULL
    int g0, n;
    int first, last;   // 1 if the leaf starts / ends its matrix (no split correction there)
    int64_t rot_off;   // first slot of the leaf's rotation buffer
    int rot_cap;       // its capacity (2 n^2 + 64 rotations)
};

// Rotations of the leaf QR iterations (phase one -> phase two).
struct LeafRot {
    double *c, *s;
    unsigned char* k;
    int* n;            // per leaf: rotations recorded (> rot_cap: overflowed)
};

// Per-level vectors indexed by global row (one entry per row of the level's
// merges) and per-merge scalars.
//   keep[i]    : 0 deflated; else the support of sorted column i after the
//                deflation rotations: 1 rows of child 1 only, 2 child 2 only,
//                3 both (rotated across the children)
//   gemmCol[p] : survivor (secular order) placed at position p of the update
//                product; positions [0,K1) have support 1, [K1,K1+Km) support
//                3, [K1+Km,K) support 2, so child-1 rows need only [0,K1+Km)
//                and child-2 rows only [K1,K)
struct LevelWS {
    double *dsort, *zsort, *dK, *zK, *wK, *lamK, *gamK, *muK, *uhat, *vv, *rot_c, *rot_s;
    int *src, *keep, *survIdx, *deflIdx, *posNew, *posDefl, *rot_j, *rot_i, *gemmCol;
    int* gemmW;        // column of W used at product position p: survIdx[gemmCol[p]]
    int *K, *nrot;     // per merge
    int* kgrp;         // per merge: K1, Km
    int* ordr;         // final ordering of an unsorted merge: rank of each value
    int* unsorted;     // per merge: 1 when the deflated poles are not ascending
    double* rho;       // per merge, after normalisation of z
    float *dhK, *dlK;  // FP32 pair of dK (dK ~ dhK + dlK, 48 bits): FP32 midpoint test and
                       // the double-float secular iterations
    float *wfK, *wlK;  // wK as an FP32 pair (wK ~ wfK + wlK)
    float* dxK;        // third part of dK: dK = dhK + dlK + dxK exactly (the double-float
                       // Cauchy kernel forms pole differences from it)
    float *ufK, *ulK;  // uhat as an FP32 pair (written by k_lowner)
};

// Per-kernel timing of a solve made with TDEIG_FLAG_PROFILE: td_prof_begin
// records an event before a launch, td_prof_end one after it (and counts the
// launch).  Events are kept in launch order.
struct TdProf {
    bool on = false;
    std::vector<cudaEvent_t> ev;
    std::vector<const char*> name;   // name at the index of each "after" event
    std::vector<std::string> note;   // optional shape of the launch, same index
    size_t n = 0;
};

// Launch count, split-product work counters and kernel timing of the calls
// made on one handle.  While a call runs, the calling thread's current record
// is its handle's own (TdCtxScope); outside calls a thread-local record takes
// the counts.  With one handle per host thread, records of different handles
// never mix.
struct TdCtx {
    long long launches = 0;
    double split_tensor_flops = 0.0;   // tensor work issued: 2 M N K per slice pair
    double split_slice_bytes = 0.0;    // algorithmic bytes of k_slice (read 8 B, write 2 s B per element)
    double split_exp_bytes = 0.0;      // algorithmic bytes of k_slice_exp (read 8 B per element)
    double split_fused_bytes = 0.0;    // algorithmic bytes of k_slice_fused (read 8 B, write 2 s B per element)
    double small_gemm_flops = 0.0;     // FP64 flops of the small-tile grouped products (k_gemm_small)
    TdProf prof;
};
TdCtx& td_ctx();
struct TdCtxScope {
    TdCtx* prev;
    explicit TdCtxScope(TdCtx* c);
    ~TdCtxScope();
};
// Raises a kernel's dynamic shared-memory limit to `bytes` on the current
// device (once per kernel, device and size).
void td_smem_attr(const void* kernel, size_t bytes);
// Number of SMs of the current device.
int td_sm_count();

void td_prof_begin(cudaStream_t st);
void td_prof_end(cudaStream_t st, const char* name);
// Attaches a note (a JSON array of numbers) to the last profiled launch.
void td_prof_note(const std::string& s);

// Host-side launchers (kernels_dc.cu).
void td_launch_scale_input(const double* d, const double* e, const int64_t* mrow0, const int64_t* mN,
                           int members, double* A, double* Bc, double* scale, int64_t R,
                           cudaStream_t st);
void td_launch_leaf(const LeafDesc* leaves, int nleaves, const double* A, const double* Bc,
                    const LeafRot& R, int* status, cudaStream_t st);
void td_launch_merge_level(const MergeDesc* M, int nmerge, int nmax, int rows, int total_tiles,
                           const LevelWS& ws, int* status, int use_hss_mask, cudaStream_t st);
// binaryVersion (major * 10 + minor) of the library's device code on the current device.
int td_binary_version(int* out);
// k_prep alone (eq. T3, sort, deflation, compaction), for the deflation stage entry point.
void td_launch_prep(const MergeDesc* M, int nmerge, const LevelWS& ws, cudaStream_t st);
// nmax: the largest merge size of the launch (bounds every K; picks the form)
void td_launch_secular(const MergeDesc* M, int nmerge, int rows, int nmax, const LevelWS& ws,
                       int* status, cudaStream_t st);
// df: the Cauchy-like matrix in double-float (split-precision solves)
void td_launch_lowner_cauchy(const MergeDesc* M, int nmerge, int rows, int kmax, const LevelWS& ws,
                             int write_qhat, cudaStream_t st, bool df = false);
// k_cauchy alone (v and, with write_qhat, the Cauchy-like matrix) from uhat.
void td_launch_cauchy(const MergeDesc* M, int nmerge, int rows, int kmax, const LevelWS& ws,
                      int write_qhat, cudaStream_t st);
// Tile-shape variants of the FP64 update product (picked per level by the autotuner).
#define TD_GEMM_VARIANTS 4
void td_gemm_tiles(int variant, int n, int* bm, int* bn);
void td_launch_update_dense(const MergeDesc* M, const int* toff, int nmerge, int total_tiles,
                            int variant, const LevelWS& ws, cudaStream_t st);
void td_launch_finish(const MergeDesc* M, int nmerge, int nmax, const LevelWS& ws, cudaStream_t st);
void td_launch_order(const MergeDesc* M, int nmerge, int nmax, const LevelWS& ws, cudaStream_t st);

// Largest total of N^2 (eigenvector entries) solved in one batched pass.
#define TD_BATCH_CHUNK ((int64_t)1 << 30)

#define TD_GEMM_BM 64
#define TD_GEMM_BN 64
#define TD_GEMM_BK 16

__host__ __device__ inline int td_cdiv(int a, int b) { return (a + b - 1) / b; }

// Merge index owning global row g (merges sorted by g0), or -1 when g lies in
// no merge of this level (rows of matrices whose tree has no merge here).
__device__ inline int td_find_merge(const MergeDesc* M, int nmerge, int g)
{
    int lo = 0, hi = nmerge - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (M[mid].g0 <= g) lo = mid; else hi = mid - 1;
    }
    if (g < M[lo].g0 || g >= M[lo].g0 + M[lo].n) return -1;
    return lo;
}

// d_k - lambda_j by Remark 1: (d_k - d_j) - gamma_j if k <= j, else
// (d_k - d_{j+1}) + mu_j.  The operands are selected, not the results, so a
// term costs one FP64 subtract and one add (x - g and x + (-g) round alike).
__device__ __forceinline__ double td_dminus(const double* d, const double* gam, const double* mu,
                                            int k, int j)
{
    const bool below = (k <= j);
    const double pole = below ? d[j] : d[j + 1];
    const double off = below ? -gam[j] : mu[j];
    return (d[k] - pole) + off;
}

// 1 / x by Newton-Raphson iteration for the reciprocal (r <- r + r (1 - x r),
// each step squaring the relative error) from the hardware's approximate FP64
// reciprocal: two steps take its ~2^-22 seed below 2^-53.  Within a few ulp,
// not correctly rounded; FP64 divides issue as long instruction sequences on
// the 1/64-rate FP64 pipe, this is five FP64 instructions.
__device__ __forceinline__ double td_recip(double x)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

__device__ __forceinline__ double td_warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double td_warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

void td_launch_stage_init(const LevelWS& ws, int K, double rho, cudaStream_t st);
