/*
 * tdeig.h -- C ABI of the GB300 (sm_103a) divide-and-conquer eigensolver for
 * symmetric tridiagonal matrices, with the accelerated (HSS) eigenvector
 * update of Li, Liao, Liu and Jiang, "New fast divide-and-conquer algorithms
 * for the symmetric tridiagonal eigenvalue problem".
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers may be host or CUDA device memory; the library detects which
 *    with cudaPointerGetAttributes.  Host arrays are staged through device
 *    workspace owned by the handle (copies are stream-ordered on the handle's
 *    stream).  Caller memory is never freed or retained by the library.
 *  - Matrices are column-major.  Q_out is N x N with leading dimension N and
 *    column j the unit eigenvector of lambda_out[j]; eigenvalues ascend.
 *    (A row-major torch tensor passed as Q_out therefore holds Q^T.)
 *  - All calls are ordered on the handle's CUDA stream and synchronise it
 *    before returning, so the status is final.  One handle per host thread.
 *  - Return value: TDEIG_OK (0) or a negative status; tdeig_strerror() gives
 *    a message.  There is no host fallback: without a usable GPU every solve
 *    returns TDEIG_ECUDA.
 */
#ifndef TDEIG_H
#define TDEIG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tdeig_ctx* tdeig_handle;

/* Eigenvector update used at merges whose deflated size exceeds
 * hss_threshold (Algorithm 1; Sec. 4.3):
 *   DENSE : the plain product diag(Q1, Q2) Qhat (standard DC);
 *   ADC1  : HSS approximation of Qhat by structured rank-revealing Schur
 *           complements (SRRSC), then Algorithm 3;
 *   ADC2  : randomized HSS construction (Algorithm 2) with the off-diagonal
 *           rank estimate of eq. (bounds), then Algorithm 3.
 * Or-ed with one precision flag for the update products (deflation, secular
 * roots, Loewner and normalisation are always FP64). */
enum {
    TDEIG_MODE_DENSE = 0,
    TDEIG_MODE_ADC1 = 1,
    TDEIG_MODE_ADC2 = 2,
    TDEIG_MODE_MASK = 0xff,
    TDEIG_PREC_FP64 = 0 << 8,     /* FP64 products */
    /* Split-precision tensor-core products (tcgen05, FP32 accumulation): the
     * dense update and Algorithm 3 from six 7-bit BF16 digit slices per operand
     * (about 42 bits), ADC2 sampling from eight (56 bits). */
    TDEIG_PREC_SPLIT = 1 << 8,
    /* Two BF16 slices (hi + lo, 16 bits) for the update and Algorithm 3;
     * sampling in FP64.  A precision-study variant: orthogonality ~1e-5. */
    TDEIG_PREC_BF16X2 = 2 << 8,
    /* Two FP16 slices (hi + lo, 22 bits; FP32 accumulation rounds); sampling in
     * FP64.  A precision-study variant. */
    TDEIG_PREC_FP16X2 = 3 << 8,
    TDEIG_PREC_MASK = 0xf << 8,
    /* DENSE (any precision) with device buffers only: capture the whole launch
     * sequence (every level of every matrix) in a CUDA graph on the first call
     * and replay it on later calls with the same sizes and buffers.  With split
     * products the launches are sized by upper bounds and read each merge's
     * deflated sizes on the device.  Ignored otherwise (the HSS modes read
     * ranks back to the host). */
    TDEIG_FLAG_GRAPH = 1 << 12,
    /* Time every kernel launch of the solve with CUDA events on the solve's
     * stream; tdeig_last_stats then lists per kernel its launches and device
     * milliseconds under "kernels".  Not combined with TDEIG_FLAG_GRAPH. */
    TDEIG_FLAG_PROFILE = 1 << 13,
    /* ADC2: record, for every node of every HSS tree, its features and the
     * rank its interpolative decompositions found (tdeig_rank_records). */
    TDEIG_FLAG_RECORD = 1 << 14,
    /* ADC2: seed the sampling rank of each HSS merge with the model given to
     * tdeig_set_rank_model (TDEIG_EINVAL when none is set): r = ceil(exp(max
     * over the merge's nodes of the prediction) - 1), clamped to [1, rank_cap].
     * When an ID of the merge stops at the sample size r + oversample with
     * more rows than that (its sampled residual is then not certified) and the
     * rank estimate of eq. (bounds) is larger than r, the merge is rebuilt with
     * the estimate; stats report "seed" per merge and "mlp_fallbacks". */
    TDEIG_FLAG_MLP_SEED = 1 << 15
};

enum {
    TDEIG_OK = 0,
    TDEIG_EINVAL = -1,    /* null pointer, N < 0, non-finite input, bad mode or option */
    TDEIG_ENOMEM = -2,    /* device workspace allocation failed */
    TDEIG_ECUDA = -3,     /* a CUDA runtime call or kernel launch failed */
    TDEIG_ENOTCONV = -4,  /* leaf QR or secular iteration hit its cap */
    TDEIG_ETIMEOUT = -5,  /* a bounded device-side wait expired */
    TDEIG_ENOTIMPL = -6   /* requested feature not built */
};

typedef struct {
    int leaf;            /* leaf size of the DC tree (paper: 25; default 32) */
    int hss_threshold;   /* use HSS when the deflated size K exceeds this (paper: 2000) */
    int hss_leaf;        /* HSS leaf block size (paper: ~200; default 128) */
    double tol;          /* HSS compression tolerance (default 1e-12) */
    int oversample;      /* p of the random sampling (paper: 10) */
    double rank_eps;     /* epsilon of the rank estimate eq. (bounds) (paper: 1e-16) */
    int rank_cap;        /* rank estimate cap (paper: 100) */
    int boundary_shift;  /* max rows a leaf boundary moves when dist < 1e-10 (paper: 5) */
    uint64_t seed;       /* seed of the Gaussian sampling matrix */
    void* cuda_stream;   /* cudaStream_t to run on; NULL = a stream owned by the handle */
} tdeig_options;

/* Fills *opt with the defaults listed above. */
void tdeig_default_options(tdeig_options* opt);

/* Creates a handle on the current CUDA device.  opt may be NULL (defaults).
 * Returns TDEIG_EINVAL for out == NULL or invalid options. */
int tdeig_create(tdeig_handle* out, const tdeig_options* opt);

/* Full eigendecomposition T = Q diag(lambda) Q^T of the symmetric tridiagonal
 * T = tridiag(e, d, e) (eq. T; Algorithm 1).
 *   d          : N diagonal entries (a_1..a_N in the paper)
 *   e          : N-1 off-diagonal entries (b_1..b_{N-1}); may be NULL if N <= 1
 *   lambda_out : N eigenvalues, ascending
 *   Q_out      : N x N column-major eigenvectors (may be NULL: eigenvalues only
 *                are still computed through the full method)
 *   mode       : TDEIG_MODE_* | TDEIG_PREC_*
 * N = 0 is a no-op; N = 1 gives lambda = d, Q = 1.  Non-finite input gives
 * TDEIG_EINVAL.  Device workspace grows inside the handle as needed. */
int tdeig_solve(tdeig_handle h, const double* d, const double* e, int64_t N,
                double* lambda_out, double* Q_out, int mode);

/* Independent problems of uneven sizes in one call.  N_each[b] is the size of
 * member b (host array).  d_cat / e_cat / lambda_cat concatenate the members'
 * arrays (e of member b has N_b - 1 entries, offsets are the prefix sums);
 * Q_cat concatenates the column-major N_b x N_b blocks (offsets: prefix sums
 * of N_b^2).  Every DC-tree level of every member runs in one launch per
 * stage. */
int tdeig_solve_batched(tdeig_handle h, int64_t batch, const int64_t* N_each,
                        const double* d_cat, const double* e_cat,
                        double* lambda_cat, double* Q_cat, int mode);

/* Frees the handle and its workspace. */
int tdeig_destroy(tdeig_handle h);

/* Static message for a status code. */
const char* tdeig_strerror(int status);

/* JSON text with per-merge statistics of the last solve on h (deflated sizes
 * K, HSS ranks, stage times).  Returns the length needed (excluding the NUL),
 * or a negative status. */
int tdeig_last_stats(tdeig_handle h, char* json_buf, size_t len);

/* ---------------------------------------------------------------------- */
/* Stage entry points of one merge, on a rank-one modified diagonal matrix */
/* M = diag(d) + rho z z^T with d strictly ascending (Theorem 1).  Used to  */
/* check the kernels stage by stage.  Pointers as above; K >= 1.           */
/* ---------------------------------------------------------------------- */

/* Secular roots (Theorem 1; Remark 1): lambda_i in (d_i, d_{i+1}) (last root
 * in (d_K, d_K + rho |z|^2]), gamma_i = lambda_i - d_i, mu_i = d_{i+1} -
 * lambda_i (mu_K = 0).  One warp per root.  TDEIG_ENOTCONV on the cap. */
int tdeig_secular(tdeig_handle h, int64_t K, const double* d, const double* z, double rho,
                  double* lambda, double* gamma, double* mu);

/* Loewner recomputation of z (eq. ev_z, with 1/rho) and the Cauchy-like
 * eigenvector matrix Qhat[k, j] = uhat_k v_j / (d_k - lambda_j) (eq. Ev-Q),
 * every d_k - lambda_j formed by Remark 1.  uhat, v: K entries; Qhat: K x K
 * column-major (may be NULL to skip it). */
int tdeig_lowner_cauchy(tdeig_handle h, int64_t K, const double* d, const double* gamma,
                        const double* mu, const double* z, double rho,
                        double* uhat, double* v, double* Qhat);

/* The same, with v and Qhat formed as split-precision solves form them
 * (eq. Ev-Q in double-float on the FP32 units: each pole as an exact triple of
 * FP32 parts, d_k - lambda_j within ~2^-47 relative however close the poles,
 * entries and norms within ~2^-44); uhat as tdeig_lowner_cauchy (FP64).
 * Arguments, layout and errors as tdeig_lowner_cauchy. */
int tdeig_lowner_cauchy_split(tdeig_handle h, int64_t K, const double* d, const double* gamma,
                              const double* mu, const double* z, double rho,
                              double* uhat, double* v, double* Qhat);

/* Split-precision product (the products of TDEIG_PREC_SPLIT / _BF16X2 /
 * _FP16X2 in isolation, not in the paper): C = op(A) op(B) with op(A) M x K,
 * op(B) K x N; A, B, C column-major FP64 with leading dimensions lda, ldb, ldc
 * (host or device); transA / transB select the transposes.  prec is one of
 * TDEIG_PREC_SPLIT, _BF16X2, _FP16X2; bits (SPLIT only, 8..56) is the number
 * of significant bits kept per operand row / column (the solver uses 40 for
 * the eigenvector products and 56 for ADC2 sampling).  C is overwritten.
 * TDEIG_EINVAL on bad sizes or arguments, TDEIG_ETIMEOUT if a bounded device
 * wait expired. */
int tdeig_split_gemm(tdeig_handle h, int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                     int transA, const double* B, int64_t ldb, int transB, double* C, int64_t ldc,
                     int prec, int bits);

/* ---------------------------------------------------------------------- */
/* Stage entry points of the integer decisions (deflation, rank estimate,   */
/* interpolative decomposition) and of the sampling generator.  Each runs   */
/* the solver's own kernel on the given inputs, so that its decisions can   */
/* be compared index for index with an independent implementation.  Array  */
/* pointers may be host or device memory as above unless stated; results   */
/* are final when the call returns.                                         */
/* ---------------------------------------------------------------------- */

/* One merge's preparation (eq. T3 and the deflation of Algorithm 1, which
 * Sec. 4.3 delegates to LAPACK's deflation; reading: Gu & Eisenstat).
 *   lam1 (n1), lam2 (n2) : the children's eigenvalues, each ascending
 *   z1 (n1) : the last row of Q1;  z2 (n2) : the first row of Q2
 *   beta    : the coupling b_k (rho = |beta|, z2 enters with sign(beta))
 * The entries are merged stably (child 1 first on ties), z is normalised
 * (rho absorbs |z|^2) and swept in ascending order against the last survivor
 * j with tau = 8 eps max(max|d|, rho max|z|): rho |z_i| <= tau deflates i;
 * otherwise, with r = hypot(z_i, z_j), c = z_i / r, s = z_j / r, |(d_i - d_j)
 * c s| <= tau rotates the pair (z_j -> 0, z_i -> r, d_j, d_i -> the diagonal
 * of G^T diag(d_j, d_i) G) and deflates j.  Outputs (any may be NULL):
 *   perm (n, int32) : sorted position p holds entry perm[p] of [lam1, lam2]
 *   d_out, z_out (n): poles and weights after the sweep (z = 0 where deflated)
 *   keep (n, int32) : 0 deflated, else the survivor's support: 1 rows of
 *                     child 1 only, 2 child 2 only, 3 both (rotated across)
 *   rho_out (host, 1), counts (host, 2): K survivors and the rotation count
 *   rot_j, rot_i (int32), rot_c, rot_s : the rotations in sweep order
 *                     (capacity n each; counts[1] are written)
 * TDEIG_EINVAL for n1 < 1, n2 < 1, n1 + n2 > 2^24 or non-finite beta. */
int tdeig_merge_deflate(tdeig_handle h, int64_t n1, int64_t n2, const double* lam1,
                        const double* lam2, const double* z1, const double* z2, double beta,
                        int32_t* perm, double* d_out, double* z_out, int32_t* keep,
                        double* rho_out, int64_t* counts, int32_t* rot_j, int32_t* rot_i,
                        double* rot_c, double* rot_s);

/* Off-diagonal rank estimate of one HSS merge (eq. bounds, with the rules of
 * Sec. 4.1): for each inner boundary b of the leaf partition, dist =
 * lambda_b - d_{b-1} = (d_b - d_{b-1}) + gamma_b (reading of eq. dist_xy);
 * a boundary with dist < 1e-10 moves by up to the handle's boundary_shift
 * rows (within its neighbours) to the largest dist; r = min(rank_cap, max_b
 * ceil(ln(16 / rank_eps) ln(8 R) / pi^2)), R = (lambda_K - d_1) / dist.
 *   d, gamma (K >= 2) : deflated poles and gaps gamma_i = lambda_i - d_i
 *   bounds (HOST int32, nl + 1, in/out): 0 = b_0 < b_1 < ... < b_nl = K
 *   r_out (HOST int32, 1) */
int tdeig_rank_estimate(tdeig_handle h, int64_t K, const double* d, const double* gamma,
                        int64_t nl, int32_t* bounds, int32_t* r_out);

/* Row interpolative decomposition Phi ~= U Phi[piv, :] (Sec. 3; Algorithm 2)
 * by Householder QR with column pivoting of Phi^T, stopped at the first k
 * with |R_kk| <= tol |R_00| (tol: the handle's option).
 *   Phi   : m x s column-major, leading dimension ldphi (1 <= m, s <= 4096;
 *           m * s doubles must fit the kernel's shared memory, else EINVAL)
 *   U     : m x rank written (leading dimension ldu), U[piv, :] = I
 *   piv   : rank int32 entries (the skeleton rows, in pivot order)
 *   rank_out (HOST int32, 1) */
int tdeig_interp_decomp(tdeig_handle h, int64_t m, int64_t s, const double* Phi, int64_t ldphi,
                        double* U, int64_t ldu, int32_t* piv, int32_t* rank_out);

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), the counter-based
 * generator of the Gaussian sampling matrix of Sec. 3: out[4t..4t+3] =
 * Philox(ctr[4t..4t+3], key[2t..2t+1]) for t < n (uint32 words). */
int tdeig_philox4x32_10(tdeig_handle h, int64_t n, const uint32_t* ctr, const uint32_t* key,
                        uint32_t* out);

/* The sampling matrix Omega of ADC2 (Sec. 3) as the solver draws it:
 * out[i + j nrow] from Philox at counter (i, j, stream_id, 0), key (seed low
 * word, seed high word), Box-Muller on the first two words with u = (x + 0.5)
 * 2^-32.  (The solver uses the DC node as stream_id.) */
int tdeig_gaussian(tdeig_handle h, int64_t nrow, int64_t ncol, uint64_t seed, uint32_t stream_id,
                   double* out);

/* The HSS eigenvector update of one merge on given generators, as a kernel
 * benchmark and stage check (Algorithm 1's "else" branch): the Cauchy-like
 * matrix Qhat[k, j] = uhat_k v_j / (d_k - lambda_j) (eq. Ev-Q, v its column
 * normalisation, lambda_j = d_j + gamma_j, every difference by Remark 1) is
 * approximated by an HSS matrix H -- ADC1: structured rank-revealing Schur
 * complements; ADC2: the rank estimate of eq. (bounds) and Algorithm 2 -- and
 * out = X H is formed by Algorithm 3.
 *   K (>= 2): size; d, gamma, mu, uhat: K entries (as tdeig_secular and
 *   tdeig_lowner_cauchy return them)
 *   P: rows of X; X, out: P x K column-major, leading dimension P
 *   mode: TDEIG_MODE_ADC1 or _ADC2 | a precision flag
 * The handle's HSS options apply (hss_leaf, tol, oversample, rank_eps,
 * rank_cap, boundary_shift, seed; the Philox stream id is 0); the HSS branch
 * is taken whatever hss_threshold says.  tdeig_last_stats then gives the
 * device milliseconds of each sub-stage ("cauchy": v and, for ADC2, the
 * sampled matrix; "hss_sample", "hss_build", "hss_mult") and the HSS record
 * (rank estimate, sample size, node ranks, moved leaf boundaries, flops). */
int tdeig_hss_apply(tdeig_handle h, int64_t K, const double* d, const double* gamma,
                    const double* mu, const double* uhat, int64_t P, const double* X, double* out,
                    int mode);

/* Architecture of the library's device code as the current device loads it:
 * *arch = major * 10 + minor (103 for sm_103a).  TDEIG_ECUDA without a GPU. */
int tdeig_binary_arch(int* arch);

/* ---------------------------------------------------------------------- */
/* Learned rank seed for ADC2 (not in the paper; it replaces the rank       */
/* estimate of eq. (bounds) as the first guess of the sampling rank r,      */
/* with that estimate kept as the fallback).                                */
/* Features of an HSS node spanning rows [s0, s1) of a merge of size n with */
/* K survivors (all logarithms of positive quantities):                     */
/*   0 log2(s1 - s0)                 block size                             */
/*   1 log10(min gap / spread)       gaps gamma_i, mu_i inside the block    */
/*   2 log10(median gap / spread)                                           */
/*   3 log10(boundary dist / spread) min over the block's boundaries of     */
/*                                   (d_b - d_{b-1}) + gamma_b (Sec. 4.1)   */
/*   4 log10(sum of uhat_i^2 in the block)   u mass                         */
/*   5 (n - K) / n                   deflated fraction                      */
/*   6 log2(K)                                                              */
/* spread = lambda_K - d_1.  Target: ln(rank + 1).                          */
/* Model: 7 -> 64 -> 64 -> 1, ReLU, weights and activations rounded to BF16,*/
/* FP32 accumulation.  Parameters (float, row-major out x in):              */
/*   W1[64][7] b1[64] W2[64][64] b2[64] W3[64] b3[1]                        */
/* Inputs are standardised with mean[7], std[7] before the first layer.     */
/* All arrays below are host or device float arrays of the stated sizes.    */
/* ---------------------------------------------------------------------- */
#define TDEIG_MLP_IN 7
#define TDEIG_MLP_HIDDEN 64
#define TDEIG_MLP_PARAMS (64 * 7 + 64 + 64 * 64 + 64 + 64 + 1)

/* y[i] = model(X[i, :]) for n samples (X row-major n x 7). */
int tdeig_mlp_forward(tdeig_handle h, const float* params, const float* mean, const float* std,
                      const float* X, int64_t n, float* y);

/* Loss 0.5 mean_i (model(X_i) - t_i)^2 and its gradient with respect to the
 * parameters (TDEIG_MLP_PARAMS floats), by the backward kernel. */
int tdeig_mlp_grad(tdeig_handle h, const float* params, const float* mean, const float* std,
                   const float* X, const float* t, int64_t n, float* loss, float* grad);

/* Adam training on the GPU: `epochs` passes over the n samples in shuffled
 * minibatches of `batch`; params holds the initial values on entry and the
 * trained ones on return; *final_loss is the loss on all samples afterwards. */
int tdeig_mlp_train(tdeig_handle h, float* params, const float* mean, const float* std,
                    const float* X, const float* t, int64_t n, int epochs, int batch, float lr,
                    uint64_t seed, float* final_loss);

/* Model used by TDEIG_FLAG_MLP_SEED (copied into the handle); params NULL
 * removes it. */
int tdeig_set_rank_model(tdeig_handle h, const float* params, const float* mean, const float* std);

/* Features (above) of nb HSS nodes of one merge: d, gamma, mu, uhat are the K
 * deflated poles, the gaps gamma_i = lambda_i - d_i and mu_i = d_{i+1} -
 * lambda_i (as tdeig_secular returns them) and the Lowner vector (host or
 * device double arrays); n >= K is the merge size; ranges (host int array,
 * 2 nb entries) holds each node's [s0, s1) with 0 <= s0 < s1 <= K; out (host
 * or device float array) receives nb x 7 features, row-major.  The median gap
 * is the centre of its bin in a histogram of 0.025-decade bins over
 * [1e-24, 100) (values outside fall in the end bins). */
int tdeig_node_features(tdeig_handle h, int64_t K, int64_t n, const double* d, const double* gamma,
                        const double* mu, const double* uhat, int64_t nb, const int* ranges,
                        float* out);

/* Records of the last solve made with TDEIG_FLAG_RECORD: 8 floats per HSS node
 * (the 7 features, then ln(rank + 1) with rank = max of the row and column ID
 * ranks); nodes whose ID stopped at the sample size are left out (their rank
 * is only a lower bound).  Copies at most cap records into buf (host) and
 * returns how many exist, or a negative status. */
int tdeig_rank_records(tdeig_handle h, float* buf, int64_t cap);

/* Largest K accepted by tdeig_secular_noalloc. */
#define TDEIG_NOALLOC_MAX_K 65536

/* Secular roots exactly as tdeig_secular computes them (the same iteration
 * from the same FP32 start, bit-identical results), but without allocating
 * any memory.  The paper has no counterpart: this entry point exists for
 * callers that cannot allocate device memory when they need the roots --
 * code that has handed all free device memory to its own pool allocator
 * (where a cudaMalloc would fail or fragment that pool), and code on a
 * latency-bound path where cudaMalloc's implicit device synchronisation is
 * not acceptable.  It needs no handle and calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *   K      : 1 <= K <= TDEIG_NOALLOC_MAX_K (65536); larger K -> TDEIG_EINVAL
 *   d, z   : K entries each, DEVICE memory of the current device (host,
 *            managed or another device's memory -> TDEIG_EINVAL)
 *   lambda, gamma, mu : K entries each, same kind of memory, written as by
 *            tdeig_secular
 *   cuda_stream : cudaStream_t to run on (NULL: the legacy default stream)
 * Scratch (the weights in FP64 and as FP32 pairs, an FP32 pair per pole and
 * a status word: 1.5 MiB in all) is a fixed array in the library's device image, held
 * by every GPU that loads the library until the process exits; each call
 * clears the status word before use.  The first call on a device, with that
 * device current, looks up the array's device address (cudaGetSymbolAddress)
 * -- make that first call before any stream capture.  All calls share the
 * array: calls whose work overlaps on the GPU (other streams or host threads)
 * race.  The call synchronises the stream and returns TDEIG_ENOTCONV if a
 * root hit the iteration cap. */
int tdeig_secular_noalloc(int64_t K, const double* d, const double* z, double rho,
                          double* lambda, double* gamma, double* mu, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* TDEIG_H */
