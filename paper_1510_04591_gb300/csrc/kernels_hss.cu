// HSS eigenvector update of the accelerated DC method (Algorithm 1, "else"
// branch): randomized HSS construction of the Cauchy-like matrix (Algorithm 2,
// ADC2) with the off-diagonal rank estimate of eq. (bounds) and Sec. 4.1, or
// structured rank-revealing Schur complements (ADC1), followed by the HSS
// matrix times general matrix product from the right (Algorithm 3).
//
// Kernels
//   k_gemm_grouped   FP64 products with gather/scatter and transposes (all the
//                    dense products of Algorithms 2 and 3)
//   k_cauchy_fill    generators D_i, B_i and Cauchy blocks from the four vectors
//   k_id             interpolative decomposition by column-pivoted Householder QR
//   k_philox_omega   Gaussian sampling matrix (Philox4x32-10 + Box-Muller)
//   k_rank_estimate  eq. (bounds) with the boundary moves and the cap of Sec. 4.1
//   k_gather_rows    skeleton rows of the children's compressed blocks
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "hss.cuh"
#include "split.cuh"
#include "mlp.cuh"

#define HSS_NT 256

// ---------------------------------------------------------------------------
// Grouped FP64 product (64 x 64 x 16 tiles, 4 x 4 outputs per thread).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(HSS_NT) k_gemm_grouped(const GemmDesc* G, int ng)
{
    __shared__ double As[16][65];
    __shared__ double Bs[16][65];
    const int bid = blockIdx.x;
    int lo = 0, hi = ng - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (G[mid].tile0 <= bid) lo = mid; else hi = mid - 1;
    }
    const GemmDesc g = G[lo];
    const int local = bid - g.tile0;
    const int tm = local % g.tiles_m, tn = local / g.tiles_m;
    const int row0 = tm * 64, col0 = tn * 64;
    if (row0 >= g.M || col0 >= g.N) return;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) acc[a][b] = 0.0;
    for (int k0 = 0; k0 < g.Kd; k0 += 16) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const int idx = threadIdx.x + HSS_NT * q;
            int r, kk;
            if (!g.transA) { r = idx & 63; kk = idx >> 6; } else { kk = idx & 15; r = idx >> 4; }
            const int i = row0 + r, k = k0 + kk;
            double va = 0.0;
            if (i < g.M && k < g.Kd) {
                if (!g.transA) {
                    const int col = g.acol ? g.acol[k] : k;
                    va = g.A[i + (int64_t)col * g.lda];
                } else {
                    va = g.A[k + (int64_t)i * g.lda];
                }
            }
            As[kk][r] = va;
            int c, kb;
            if (!g.transB) { kb = idx & 15; c = idx >> 4; } else { c = idx & 63; kb = idx >> 6; }
            const int j = col0 + c, kg = k0 + kb;
            double vb = 0.0;
            if (j < g.N && kg < g.Kd)
                vb = g.transB ? g.B[j + (int64_t)kg * g.ldb] : g.B[kg + (int64_t)j * g.ldb];
            Bs[kb][c] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; kk++) {
            double av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; a++) av[a] = As[kk][tx + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; b++) bv[b] = Bs[kk][ty + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; a++)
#pragma unroll
                for (int b = 0; b < 4; b++) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int b = 0; b < 4; b++) {
        const int j = col0 + ty + 16 * b;
        if (j >= g.N) continue;
        double* out = g.C + (int64_t)(g.ccol ? g.ccol[j] : j) * g.ldc;
#pragma unroll
        for (int a = 0; a < 4; a++) {
            const int i = row0 + tx + 16 * a;
            if (i < g.M) out[i] = g.beta != 0.0 ? g.alpha * acc[a][b] + g.beta * out[i]
                                                : g.alpha * acc[a][b];
        }
    }
}

// Small problems (the HSS construction's products: sides of one or two ranks,
// a few tens to a hundred and some): 16 x 16 output tiles, one output per
// thread, k in chunks of 32 through shared memory.  The FP64 pipe (2 lanes per
// clock per SM) bounds each CTA, so the 64 x 64 tiles above, padded to the
// tile and few in number, left most SMs idle while each busy one worked for
// ~0.1 ms; small tiles spread the same work over the whole GPU and pad less.
#define GT_T 16
#define GT_K 32
__global__ void __launch_bounds__(GT_T * GT_T) k_gemm_small(const GemmDesc* G, int ng)
{
    __shared__ double As[GT_K][GT_T + 1];
    __shared__ double Bs[GT_K][GT_T + 1];
    const int bid = blockIdx.x;
    int lo = 0, hi = ng - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (G[mid].tile0 <= bid) lo = mid; else hi = mid - 1;
    }
    const GemmDesc g = G[lo];
    const int local = bid - g.tile0;
    const int row0 = (local % g.tiles_m) * GT_T, col0 = (local / g.tiles_m) * GT_T;
    if (row0 >= g.M || col0 >= g.N) return;
    const int tx = threadIdx.x & (GT_T - 1), ty = threadIdx.x / GT_T;
    double acc = 0.0;
    for (int k0 = 0; k0 < g.Kd; k0 += GT_K) {
#pragma unroll
        for (int q = 0; q < 2; q++) {
            const int idx = threadIdx.x + GT_T * GT_T * q;   // 512 entries per operand
            int r, kk;
            if (!g.transA) { r = idx & (GT_T - 1); kk = idx / GT_T; } else { kk = idx & (GT_K - 1); r = idx / GT_K; }
            const int i = row0 + r, k = k0 + kk;
            double va = 0.0;
            if (i < g.M && k < g.Kd) {
                if (!g.transA) {
                    const int col = g.acol ? g.acol[k] : k;
                    va = g.A[i + (int64_t)col * g.lda];
                } else {
                    va = g.A[k + (int64_t)i * g.lda];
                }
            }
            As[kk][r] = va;
            int c, kb;
            if (!g.transB) { kb = idx & (GT_K - 1); c = idx / GT_K; } else { c = idx & (GT_T - 1); kb = idx / GT_T; }
            const int j = col0 + c, kg = k0 + kb;
            double vb = 0.0;
            if (j < g.N && kg < g.Kd)
                vb = g.transB ? g.B[j + (int64_t)kg * g.ldb] : g.B[kg + (int64_t)j * g.ldb];
            Bs[kb][c] = vb;
        }
        __syncthreads();
        const int kn = min(GT_K, g.Kd - k0);
#pragma unroll 8
        for (int kk = 0; kk < kn; kk++) acc = fma(As[kk][tx], Bs[kk][ty], acc);
        __syncthreads();
    }
    const int i = row0 + tx, j = col0 + ty;
    if (i < g.M && j < g.N) {
        double* out = g.C + (int64_t)(g.ccol ? g.ccol[j] : j) * g.ldc;
        out[i] = g.beta != 0.0 ? g.alpha * acc + g.beta * out[i] : g.alpha * acc;
    }
}

double hss_launch_gemm(const std::vector<GemmDesc>& gin, GemmDesc* dev, cudaStream_t st)
{
    // every problem small: 16 x 16 tiles; else the 64 x 64 tiles
    bool small = true;
    for (const GemmDesc& d : gin)
        if (d.M > 0 && d.N > 0 && (d.M > 256 || d.N > 256)) small = false;
    const int T = small ? GT_T : 64;
    std::vector<GemmDesc> g;
    g.reserve(gin.size());
    int tiles = 0;
    double flops = 0.0;
    for (GemmDesc d : gin) {
        if (d.M <= 0 || d.N <= 0) continue;
        d.tiles_m = td_cdiv(d.M, T);
        d.tile0 = tiles;
        tiles += d.tiles_m * td_cdiv(d.N, T);
        flops += 2.0 * d.M * d.N * d.Kd;
        g.push_back(d);
    }
    if (g.empty()) return 0.0;
    cudaMemcpyAsync(dev, g.data(), g.size() * sizeof(GemmDesc), cudaMemcpyHostToDevice, st);
    td_prof_begin(st);
    if (small) k_gemm_small<<<tiles, GT_T * GT_T, 0, st>>>(dev, (int)g.size());
    else k_gemm_grouped<<<tiles, HSS_NT, 0, st>>>(dev, (int)g.size());
    td_prof_end(st, small ? "k_gemm_small" : "k_gemm_grouped");
    if (small) td_ctx().small_gemm_flops += flops;
    return flops;
}

// ---------------------------------------------------------------------------
// Cauchy-like blocks from the generators (Sec. 4.1: D_i and B_i are recomputed
// from the four vectors rather than read from the full matrix).
// ---------------------------------------------------------------------------
__global__ void k_cauchy_fill(const FillDesc* F, int nf)
{
    const int bid = blockIdx.x;
    int lo = 0, hi = nf - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (F[mid].tile0 <= bid) lo = mid; else hi = mid - 1;
    }
    const FillDesc f = F[lo];
    const int local = bid - f.tile0;
    const int ta = local % f.tiles_r, tb = local / f.tiles_r;
    const int a = ta * 32 + (threadIdx.x & 31);
    if (a >= f.nr) return;
    const int k = f.rows ? f.rows[a] : f.r0 + a;
    const double uk = f.uhat[k];
    for (int bb = threadIdx.x >> 5; bb < 32; bb += HSS_NT / 32) {
        const int b = tb * 32 + bb;
        if (b >= f.nc) break;
        const int j = f.cols ? f.cols[b] : f.c0 + b;
        f.out[a + (int64_t)b * f.ld] = uk * f.v[j] / td_dminus(f.d, f.gam, f.mu, k, j);
    }
}

static void launch_fill(std::vector<FillDesc>& F, FillDesc* dev, cudaStream_t st)
{
    std::vector<FillDesc> f;
    int tiles = 0;
    for (FillDesc d : F) {
        if (d.nr <= 0 || d.nc <= 0) continue;
        d.tiles_r = td_cdiv(d.nr, 32);
        d.tile0 = tiles;
        tiles += d.tiles_r * td_cdiv(d.nc, 32);
        f.push_back(d);
    }
    if (f.empty()) return;
    cudaMemcpyAsync(dev, f.data(), f.size() * sizeof(FillDesc), cudaMemcpyHostToDevice, st);
    td_prof_begin(st);
    k_cauchy_fill<<<tiles, HSS_NT, 0, st>>>(dev, (int)f.size());
    td_prof_end(st, "k_cauchy_fill");
}

// ---------------------------------------------------------------------------
// Row gather: dst[a, :] = src[piv[a], :]
// ---------------------------------------------------------------------------
__global__ void k_gather_rows(const GatherDesc* Gd, int ng)
{
    const GatherDesc g = Gd[blockIdx.y];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < g.nr * g.ncols; t += gridDim.x * blockDim.x) {
        const int a = t % g.nr, c = t / g.nr;
        g.dst[a + (int64_t)c * g.ldd] = g.src[g.piv[a] + (int64_t)c * g.lds];
    }
}

static void launch_gather(const std::vector<GatherDesc>& G, GatherDesc* dev, cudaStream_t st)
{
    std::vector<GatherDesc> g;
    for (auto& d : G)
        if (d.nr > 0 && d.ncols > 0) g.push_back(d);
    if (g.empty()) return;
    cudaMemcpyAsync(dev, g.data(), g.size() * sizeof(GatherDesc), cudaMemcpyHostToDevice, st);
    td_prof_begin(st);
    k_gather_rows<<<dim3(8, (unsigned)g.size()), HSS_NT, 0, st>>>(dev, (int)g.size());
    td_prof_end(st, "k_gather_rows");
}

// Row stride of the ID's matrix in shared memory: the smallest ld >= m with
// ld = 8 (mod 16), so that the update's four row phases of eight neighbouring
// columns fall in distinct double-word banks (two wavefronts per warp).
__host__ __device__ __forceinline__ int id_ld(int m) { return m + ((24 - (m & 15)) & 15); }

// ---------------------------------------------------------------------------
// Interpolative decomposition (Sec. 3): Householder QR with column pivoting of
// Phi^T (s x m; its columns are the rows of Phi), stopped at the first k with
// |R_kk| <= tol |R_00|.  With R = [R11 R12], T = R11^{-1} R12 and the pivot
// order P, U = P [I; T^T] so that Phi ~= U Phi[piv, :].  One CTA per matrix;
// Phi^T lives in shared memory row-major (A[i*m + j], i < s, j < m).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(HSS_NT) k_id(const IdDesc* D, int nd, double tol)
{
    extern __shared__ double sm[];
    __shared__ long long redb[HSS_NT / 32];
    __shared__ int redi[HSS_NT / 32];
    const IdDesc g = D[blockIdx.x];
    const int m = g.m, s = g.s;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int q4 = tid & 3;
    const int ld = id_ld(m);              // row stride of A (see id_ld)
    double* A = sm;                       // s x m, rows ld apart
    double* nrm = A + (size_t)s * ld;     // m: squared norm of the rows below the current step
    double* ref = nrm + m;                // m: that norm when last computed exactly
    int* perm = (int*)(ref + m);          // m
    for (int t = tid; t < s * m; t += HSS_NT) {
        const int j = t % m, i = t / m;
        A[i * ld + j] = g.Phi[j + (int64_t)i * g.ldphi];
    }
    __syncthreads();
    for (int j = tid; j < m; j += HSS_NT) {
        double a = 0.0;
        for (int i = 0; i < s; i++) a += A[i * ld + j] * A[i * ld + j];
        nrm[j] = a;
        ref[j] = a;
        perm[j] = j;
    }
    __syncthreads();
    // Four barriers per step: after the pivot's partial maxima, after the
    // column swap, after the Householder scalars, after the update.  Scalar
    // FP64 work (the pivot column's norm, square root, divide) is done by one
    // warp and shared through shared memory: repeated by all 256 threads it
    // cost several times the update itself on the 1/64-rate FP64 pipe, and the
    // pivot search compares the non-negative norms as integers for the same
    // reason.  The remaining column norms are downdated and, as in LAPACK's
    // xGEQP3, recomputed only when the downdate has fallen below sqrt(eps) of
    // the last exact value (norms serve the pivot choice only); the pivot
    // column's norm is always computed exactly.
    __shared__ double s_par[3];
    __shared__ int s_stop;
    const int kmax = min(s, m);
    double r00 = 0.0;
    int rank = kmax;
    for (int k = 0; k < kmax; k++) {
        // pivot: largest remaining column norm, lowest index on ties
        long long best = -1;
        int bi = k;
        for (int j = k + tid; j < m; j += HSS_NT) {
            const long long v = __double_as_longlong(nrm[j]);
            if (v > best) { best = v; bi = j; }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { redb[wid] = best; redi[wid] = bi; }
        __syncthreads();
        best = redb[0];
        bi = redi[0];
        for (int w = 1; w < HSS_NT / 32; w++)
            if (redb[w] > best || (redb[w] == best && redi[w] < bi)) { best = redb[w]; bi = redi[w]; }
        const int p = bi;
        if (k == 0) {
            if (best <= 0) { rank = 0; break; }   // zero matrix
            if (tid == 0) r00 = sqrt(__longlong_as_double(best));   // exact first pivot norm
        }
        if (p != k) {
            for (int i = tid; i < s; i += HSS_NT) {
                double t = A[i * ld + k]; A[i * ld + k] = A[i * ld + p]; A[i * ld + p] = t;
            }
            if (tid == 0) {
                double t = nrm[k]; nrm[k] = nrm[p]; nrm[p] = t;
                t = ref[k]; ref[k] = ref[p]; ref[p] = t;
                int u = perm[k]; perm[k] = perm[p]; perm[p] = u;
            }
        }
        __syncthreads();
        if (wid == 0) {
            double a = 0.0;
            for (int i = k + lane; i < s; i += 32) a += A[i * ld + k] * A[i * ld + k];
            a = td_warp_sum(a);
            if (lane == 0) {
                const double xn = sqrt(a);
                const double x0 = A[k * ld + k];
                const double alpha = (x0 >= 0.0) ? -xn : xn;
                s_stop = xn <= tol * r00;
                s_par[0] = td_recip(alpha * (alpha - x0));   // beta (Newton reciprocal, a few ulp)
                s_par[1] = x0 - alpha;                     // first entry of the Householder vector
                s_par[2] = alpha;
            }
        }
        __syncthreads();
        if (s_stop) { rank = k; break; }
        const double beta = s_par[0], v0 = s_par[1];
        // Four lanes per column (lane q of a group takes rows k+1+q, k+5+q, ...;
        // the dot product's partial sums are combined by shuffles): one lane per
        // column left the SM's FP64 units partly idle and each column's sum one
        // long dependent chain.  Whole warps iterate together (shuffles).
        for (int base = k + 1; base < m; base += HSS_NT / 4) {
            const int j = base + (tid >> 2);
            const bool act = j < m;
            double dot = 0.0;
            if (act) {
                if (q4 == 0) dot = v0 * A[k * ld + j];
                for (int i = k + 1 + q4; i < s; i += 4) dot = fma(A[i * ld + k], A[i * ld + j], dot);
            }
            dot += __shfl_xor_sync(0xffffffffu, dot, 1);
            dot += __shfl_xor_sync(0xffffffffu, dot, 2);
            double akj = 0.0;
            if (act) {
                const double f = beta * dot;
                if (q4 == 0) {
                    akj = A[k * ld + j] - f * v0;
                    A[k * ld + j] = akj;
                }
                for (int i = k + 1 + q4; i < s; i += 4) A[i * ld + j] -= f * A[i * ld + k];
            }
            int rec = 0;
            double nn = 0.0;
            if (act && q4 == 0) {
                nn = nrm[j] - akj * akj;
                rec = !(nn > 1.4901161193847656e-8 * ref[j]);   // sqrt(2^-52)
            }
            rec = __shfl_sync(0xffffffffu, rec, lane & ~3);
            if (__any_sync(0xffffffffu, rec)) {
                // exact norm of the rows below k (each lane its own rows, updated above)
                double a = 0.0;
                if (act && rec)
                    for (int i = k + 1 + q4; i < s; i += 4) a = fma(A[i * ld + j], A[i * ld + j], a);
                a += __shfl_xor_sync(0xffffffffu, a, 1);
                a += __shfl_xor_sync(0xffffffffu, a, 2);
                if (rec) {
                    nn = a;
                    if (act && q4 == 0) ref[j] = a;
                }
            }
            if (act && q4 == 0) nrm[j] = nn;
        }
        __syncthreads();
        if (tid == 0) A[k * ld + k] = s_par[2];   // column k is read by no one until the end
    }
    __syncthreads();
    // T = R11^{-1} R12 in place (columns rank..m-1), back substitution by groups
    // of four lanes per column (each lane a quarter of every row's sum, combined
    // by shuffles), with the diagonal's reciprocals taken once: one lane per
    // column left most of the SM's FP64 units idle and spent ~40 % of the work
    // on divides
    double* rdiag = nrm;   // the column norms are no longer needed
    for (int i = tid; i < rank; i += HSS_NT) rdiag[i] = 1.0 / A[i * ld + i];
    __syncthreads();
    {
        const int q = lane & 3;
        const unsigned gmask = 0xFu << (lane & ~3);
        const int ncol = m - rank;
        // whole warps iterate together (the group shuffles need all four lanes)
        for (int base = 0; base < ncol; base += HSS_NT / 4) {
            const int jj = base + (tid >> 2);
            const bool act = jj < ncol;
            const int j = rank + (act ? jj : 0);
            for (int i = rank - 1; i >= 0; i--) {
                double t = 0.0;
                if (act)
                    for (int l = i + 1 + q; l < rank; l += 4) t = fma(A[i * ld + l], A[l * ld + j], t);
                t += __shfl_xor_sync(gmask, t, 1);
                t += __shfl_xor_sync(gmask, t, 2);
                if (act && q == 0) A[i * ld + j] = (A[i * ld + j] - t) * rdiag[i];
                __syncwarp();
            }
        }
    }
    __syncthreads();
    for (int t = tid; t < m * rank; t += HSS_NT) {
        const int row = t % m, c = t / m;   // row = position in pivot order
        const double val = (row < rank) ? (row == c ? 1.0 : 0.0) : A[c * ld + row];
        g.U[perm[row] + (int64_t)c * g.ldu] = val;
    }
    for (int c = tid; c < rank; c += HSS_NT) {
        const int pr = perm[c];
        g.out_piv[c] = pr;
        g.out_idx[c] = g.rowmap ? (pr < g.n1 ? g.rowmap[pr] : g.rowmap2[pr - g.n1]) : g.rowbase + pr;
    }
    if (tid == 0) *g.out_rank = rank;
}

static size_t id_smem(int s, int m) { return (size_t)s * id_ld(m) * 8 + (size_t)m * 20 + (size_t)s * 8 + 64; }

int hss_launch_id(const IdDesc* dev, int nd, int smax, int mmax, double tol, cudaStream_t st)
{
    const size_t sm = id_smem(smax, mmax);
    if (sm > 220 * 1024) return TDEIG_EINVAL;
    if (nd <= 0) return TDEIG_OK;
    td_smem_attr((const void*)k_id, 220 * 1024);
    td_prof_begin(st);
    k_id<<<(unsigned)nd, HSS_NT, sm, st>>>(dev, nd, tol);
    td_prof_end(st, "k_id");
    return TDEIG_OK;
}

// ---------------------------------------------------------------------------
// Gaussian sampling matrix: Omega[i, j] from Philox4x32-10 (Salmon, Moraes,
// Dror, Shaw, SC'11) with counter (i, j, stream, 0) and key (seed low, seed
// high); Box-Muller on the first two output words, u = (x + 0.5) 2^-32.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
    const unsigned M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        const unsigned hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const unsigned hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += W0;
        k.y += W1;
    }
    return c;
}

__global__ void k_philox_omega(double* Om, int K, int s, unsigned long long seed, unsigned stream)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)K * s) return;
    const int i = (int)(t % K), j = (int)(t / K);
    const uint4 r = philox4x32_10(make_uint4((unsigned)i, (unsigned)j, stream, 0u),
                                  make_uint2((unsigned)(seed & 0xffffffffull), (unsigned)(seed >> 32)));
    const double u1 = ((double)r.x + 0.5) * 2.3283064365386963e-10;
    const double u2 = ((double)r.y + 0.5) * 2.3283064365386963e-10;
    Om[t] = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

// Raw Philox words for n counters (the stage entry point tdeig_philox4x32_10).
__global__ void k_philox_words(const unsigned* ctr, const unsigned* key, unsigned* out, int64_t n)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const uint4 r = philox4x32_10(make_uint4(ctr[4 * t], ctr[4 * t + 1], ctr[4 * t + 2], ctr[4 * t + 3]),
                                  make_uint2(key[2 * t], key[2 * t + 1]));
    out[4 * t] = r.x;
    out[4 * t + 1] = r.y;
    out[4 * t + 2] = r.z;
    out[4 * t + 3] = r.w;
}

void hss_launch_philox_words(const unsigned* ctr, const unsigned* key, unsigned* out, int64_t n,
                             cudaStream_t st)
{
    if (n <= 0) return;
    td_prof_begin(st);
    k_philox_words<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(ctr, key, out, n);
    td_prof_end(st, "k_philox_words");
}

void hss_launch_gaussian(double* Om, int K, int s, unsigned long long seed, unsigned stream,
                         cudaStream_t st)
{
    const int64_t tot = (int64_t)K * s;
    if (tot <= 0) return;
    td_prof_begin(st);
    k_philox_omega<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(Om, K, s, seed, stream);
    td_prof_end(st, "k_philox_omega");
}

// ---------------------------------------------------------------------------
// Off-diagonal rank estimate (eq. bounds, Sec. 4.1).  At the boundary b between
// neighbouring leaf segments dist = lambda_b - d_{b-1} = (d_b - d_{b-1}) +
// gamma_b (d in the left segment, lambda in the right one); boundaries with
// dist < 1e-10 move by up to `shift` rows to the largest dist;
// r = min(cap, max_b ceil(ln(16/eps) ln(8R)/pi^2)), R = (lambda_K - d_1)/dist.
// One thread per merge (sequential over boundaries, as the moves chain).
// ---------------------------------------------------------------------------
__global__ void k_rank_estimate(const RankDesc* Rd, int nr, double eps, int cap, int shift)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nr) return;
    const RankDesc R = Rd[t];
    const double* d = R.d;
    const double* gam = R.gam;
    const double span = (d[R.K - 1] + gam[R.K - 1]) - d[0];
    int r = 1;
    for (int sidx = 1; sidx < R.nl; sidx++) {
        int b = R.bounds[sidx];
        double dist = (d[b] - d[b - 1]) + gam[b];
        if (dist < 1e-10) {
            int best_b = b;
            double best = dist;
            const int lo = R.bounds[sidx - 1] + 1, hi = R.bounds[sidx + 1] - 1;
            for (int s = 1; s <= shift; s++) {
                for (int side = 0; side < 2; side++) {
                    const int cand = side ? b + s : b - s;
                    if (cand >= lo && cand <= hi) {
                        const double dc = (d[cand] - d[cand - 1]) + gam[cand];
                        if (dc > best) { best_b = cand; best = dc; }
                    }
                }
            }
            R.bounds[sidx] = best_b;
            dist = best;
        }
        int rb = cap;
        if (dist > 0.0) {
            const double Rr = span / dist;
            if (isfinite(Rr)) rb = (int)ceil(log(16.0 / eps) * log(8.0 * Rr) / (M_PI * M_PI));
        }
        r = max(r, rb);
    }
    *R.r_out = min(r, cap);
}

void hss_launch_rank_estimate(const RankDesc* dev, int nr, double eps, int cap, int shift,
                              cudaStream_t st)
{
    if (nr <= 0) return;
    td_prof_begin(st);
    k_rank_estimate<<<td_cdiv(nr, 64), 64, 0, st>>>(dev, nr, eps, cap, shift);
    td_prof_end(st, "k_rank_estimate");
}

// ---------------------------------------------------------------------------
// ADC1 compression (structured rank-revealing Schur complements, the paper's
// SRRSC reading): complete-pivoting elimination on the generator form of one
// HSS block row / column C[a, b] = g_a h_b / (d - lambda).  Each elimination
// step keeps the Schur complement Cauchy-like: with pivot (p, q),
//   g_a <- g_a - (S_aq / S_pq) g_p,   h_b <- h_b - (S_pb / S_pq) h_q,
// S entries recomputed from the generators and Remark 1 differences in FP64.
// The pivot search reads FP32 magnitudes |1/(d - lambda)| materialised once
// per block, so only the search is approximate (a near-maximal pivot is still
// a complete-pivoting choice).  Stop at |S_pq| <= tol |first pivot|.  With the
// multipliers l_a (row a's elimination multipliers) and L11 those of the pivot
// rows, U = C[:, pc] C[pr, pc]^{-1} = l L11^{-1}, so C ~= U C[pr, :].
// One CTA per block.
// ---------------------------------------------------------------------------
#define SR_NT 512
#define SR_MAXM 512
#define SR_MAXK 256

__device__ __forceinline__ int sr_row(const SrrscDesc& g, int a)
{
    return a < g.n1 ? g.map1[a] : (g.map2 ? g.map2[a - g.n1] : g.base + a);
}

__device__ __forceinline__ int sr_col(const SrrscDesc& g, int b)
{
    return b < g.s0 ? b : b + (g.s1 - g.s0);
}

__device__ __forceinline__ double sr_diff(const SrrscDesc& g, int r, int c)
{
    return g.side == 0 ? td_dminus(g.d, g.gam, g.mu, r, c) : td_dminus(g.d, g.gam, g.mu, c, r);
}

// Pole data of an index x for the pivot search, in FP32: [dh, dl] of d_x (an
// FP32 pair), [dh, dl] of d_x and of d_x+1 and the Remark 1 offsets -gamma_x,
// mu_x (for |d_k - lambda_x|).
__device__ __forceinline__ void sr_pole_f32(const SrrscDesc& g, int x, float* o)
{
    const double dx = g.d[x];
    const float h = __double2float_rn(dx);
    o[0] = h;
    o[1] = __double2float_rn(dx - (double)h);
    o[2] = o[0];
    o[3] = o[1];
    const bool nx = x + 1 < g.K;
    const double d1 = nx ? g.d[x + 1] : 0.0;
    const float h1 = __double2float_rn(d1);
    o[4] = h1;
    o[5] = __double2float_rn(d1 - (double)h1);
    o[6] = __double2float_rn(-g.gam[x]);
    o[7] = __double2float_rn(g.mu[x]);
}

// d_K - lambda_J in FP32 (Remark 1), K's pair (kh, kl), J's pole data J.
__device__ __forceinline__ float sr_diff_f32(float kh, float kl, int kidx, const float* J, int jidx)
{
    const bool below = kidx <= jidx;
    const float ph = below ? J[2] : J[4], pl = below ? J[3] : J[5];
    return ((kh - ph) + (kl - pl)) + (below ? J[6] : J[7]);
}

__global__ void __launch_bounds__(SR_NT) k_srrsc(const SrrscDesc* D, double tol, int* status)
{
    __shared__ float redv[SR_NT / 32];
    __shared__ int redi[SR_NT / 32];
    __shared__ int s_p, s_q, s_stop;
    __shared__ double s_spq;
    __shared__ int s_pr[SR_MAXK];
    __shared__ int s_rowpos[SR_MAXM];
    // rows' pole data, global indices, FP32 generators and active flags
    __shared__ float s_row[SR_MAXM][8];
    __shared__ int s_ridx[SR_MAXM];
    __shared__ float s_gf[SR_MAXM];
    __shared__ unsigned char s_act[SR_MAXM];
    const SrrscDesc g = D[blockIdx.x];
    const int m = g.m, nc = g.K - (g.s1 - g.s0);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    float* const ctab = g.invd;   // per column: its pole data (8 floats)
    for (int a = tid; a < m; a += SR_NT) {
        const int ra = sr_row(g, a);
        const double gv = g.side == 0 ? g.uh[ra] : g.v[ra];
        g.g[a] = gv;
        g.gf[a] = (float)gv;
        g.actr[a] = 1;
        s_rowpos[a] = -1;
        s_ridx[a] = ra;
        s_gf[a] = (float)gv;
        s_act[a] = 1;
        sr_pole_f32(g, ra, s_row[a]);
    }
    for (int b = tid; b < nc; b += SR_NT) {
        const int cb = sr_col(g, b);
        const double hv = g.side == 0 ? g.v[cb] : g.uh[cb];
        g.h[b] = hv;
        g.hf[b] = (float)hv;
        g.actc[b] = 1;
        float o[8];
        sr_pole_f32(g, cb, o);
        float4* c4 = reinterpret_cast<float4*>(ctab + (size_t)8 * b);
        c4[0] = make_float4(o[0], o[1], o[2], o[3]);
        c4[1] = make_float4(o[4], o[5], o[6], o[7]);
    }
    __syncthreads();
    const int kmax = min(g.kcap, min(m, nc));
    double first = 0.0;
    int rank = 0;
    for (int t = 0; t < kmax; t++) {
        // Pivot: the largest |g_a h_b / (d - lambda)| over the active block, in
        // FP32 with the differences formed on the fly (Remark 1, FP32 pairs of
        // the poles): each thread owns columns and sweeps the rows held in
        // shared memory.  (A stored m x ncols table of 1/|d - lambda| re-read
        // every step kept the kernel waiting on memory.)  The pivot's entry is
        // then formed in FP64.  Ties go to the lowest row-major index.
        float best = -1.0f;
        int bi = 0x7fffffff;
        for (int b = tid; b < nc; b += SR_NT) {
            if (!g.actc[b]) continue;
            const float hb = fabsf(g.hf[b]);
            const int cb = sr_col(g, b);
            const float4* c4 = reinterpret_cast<const float4*>(ctab + (size_t)8 * b);
            const float4 u0 = c4[0], u1 = c4[1];
            const float C[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
            for (int a = 0; a < m; a++) {
                if (!s_act[a]) continue;
                const float dv = g.side == 0 ? sr_diff_f32(s_row[a][0], s_row[a][1], s_ridx[a], C, cb)
                                             : sr_diff_f32(C[0], C[1], cb, s_row[a], s_ridx[a]);
                const float val = fabsf(s_gf[a]) * hb / fabsf(dv);
                const int idx = a * nc + b;
                if (val > best || (val == best && idx < bi)) { best = val; bi = idx; }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) { redv[wid] = best; redi[wid] = bi; }
        __syncthreads();
        if (tid == 0) {
            float bb = -1.0f;
            int ib = 0x7fffffff;
            for (int w = 0; w < SR_NT / 32; w++)
                if (redv[w] > bb || (redv[w] == bb && redi[w] < ib)) { bb = redv[w]; ib = redi[w]; }
            int stop = (ib == 0x7fffffff);
            double spq = 0.0;
            if (!stop) {
                const int p = ib / nc, q = ib - p * nc;
                spq = g.g[p] * g.h[q] / sr_diff(g, sr_row(g, p), sr_col(g, q));
                if (t == 0) first = fabs(spq);
                stop = (first == 0.0 || !(fabs(spq) > tol * first));
                s_p = p;
                s_q = q;
                if (!stop) { s_pr[t] = p; s_rowpos[p] = t; }
            }
            s_spq = spq;
            s_stop = stop;
        }
        __syncthreads();
        if (s_stop) break;
        const int p = s_p, q = s_q;
        const double spq = s_spq, gp = g.g[p], hq = g.h[q];
        const int rp = sr_row(g, p), cq = sr_col(g, q);
        // Schur-complement update of the generators.  Divides are Newton
        // reciprocals (td_recip, a few ulp) and the pivot's reciprocal is taken
        // once: IEEE divides, two per row or column and step, issued as long
        // sequences on the 1/64-rate FP64 pipe and bound the kernel.
        const double rspq = td_recip(spq), hq_spq = hq * rspq;
        for (int a = tid; a < m; a += SR_NT) {
            if (!g.actr[a]) continue;
            if (a == p) { g.mult[(size_t)a * g.kcap + t] = 1.0; continue; }
            const double l = g.g[a] * hq_spq * td_recip(sr_diff(g, sr_row(g, a), cq));   // s_aq / s_pq
            g.mult[(size_t)a * g.kcap + t] = l;
            const double ga = g.g[a] - l * gp;
            g.g[a] = ga;
            g.gf[a] = (float)ga;
            s_gf[a] = (float)ga;
        }
        for (int b = tid; b < nc; b += SR_NT) {
            if (!g.actc[b] || b == q) continue;
            const double spb = gp * g.h[b] * td_recip(sr_diff(g, rp, sr_col(g, b)));
            const double hb = g.h[b] - spb * hq_spq;
            g.h[b] = hb;
            g.hf[b] = (float)hb;
        }
        __syncthreads();
        if (tid == 0) { g.actr[p] = 0; g.actc[q] = 0; s_act[p] = 0; }
        __syncthreads();
        rank = t + 1;
    }
    if (tid == 0 && rank == g.kcap && kmax == g.kcap) atomicOr(status, TD_STATUS_BADRANK);
    // U rows: pivot rows are unit rows; the others solve x L11 = l_a backwards.
    for (int a = tid; a < m; a += SR_NT) {
        const int pos = s_rowpos[a];
        if (pos >= 0 && pos < rank) {
            for (int c = 0; c < rank; c++) g.U[a + (size_t)c * g.ldu] = (c == pos) ? 1.0 : 0.0;
            continue;
        }
        for (int c = rank - 1; c >= 0; c--) {
            double x = g.mult[(size_t)a * g.kcap + c];
            for (int i = c + 1; i < rank; i++)
                x -= g.U[a + (size_t)i * g.ldu] * g.mult[(size_t)s_pr[i] * g.kcap + c];
            g.U[a + (size_t)c * g.ldu] = x;
        }
    }
    for (int c = tid; c < rank; c += SR_NT) {
        g.out_piv[c] = s_pr[c];
        g.out_idx[c] = sr_row(g, s_pr[c]);
    }
    if (tid == 0) *g.out_rank = rank;
}

// ---------------------------------------------------------------------------
// Host orchestration
// ---------------------------------------------------------------------------
namespace {

struct HNode {
    int r0 = 0, r1 = 0;          // leaf index range
    int kU = 0, kV = 0;
    double *U = nullptr, *V = nullptr;
    int ldU = 0;
    double *Phi = nullptr, *Theta = nullptr;
    int ldPhi = 0;
    int *I = nullptr, *J = nullptr, *pivI = nullptr, *pivJ = nullptr, *rk = nullptr;
    double *Ystk = nullptr, *Zstk = nullptr;   // parents: stacked Yhat / Zhat of the children
    double* B = nullptr;                       // non-root: kU x kV(sibling), ld s
    double* D = nullptr;                       // leaves: m x m, ld mcap
};

struct HMerge {
    int mi = 0, K = 0, n = 0, L = 0, r = 0, s = 0, mcap = 0, node_id = 0;
    int r_est = 0;     // rank estimate of eq. (bounds)
    int seed = 0;      // 0 estimate, 1 learned seed, 2 learned seed rejected -> estimate
    size_t feat0 = 0;  // first node of this merge in the feature array
    std::vector<int> bounds;
    std::vector<HNode> nodes;
    double *Om = nullptr, *Y = nullptr, *Z = nullptr;
    int* leaf_of = nullptr;   // HSS leaf of every row (masked split sampling)
    std::vector<double*> G, F;      // per level 1..L: n x 2^l s, ld n
    const double *d, *gam, *mu, *uh, *v, *qhat;
    const int *surv, *posNew;
    double *W, *qout;
    int* dev_bounds = nullptr;
    int* dev_r = nullptr;
};

inline int hidx(int l, int q) { return (1 << l) - 1 + q; }

struct Bump {
    char* base;
    size_t off, cap;
    template <class T> T* take(size_t n)
    {
        off = (off + 255) & ~(size_t)255;
        T* p = (T*)(base + off);
        off += n * sizeof(T);
        return p;
    }
};

}  // namespace

void hss_free(HssWS& w)
{
    if (w.base) cudaFree(w.base);
    w.base = nullptr;
    w.cap = 0;
}

static int grow(HssWS& w, size_t bytes, cudaStream_t st)
{
    if (bytes <= w.cap) return TDEIG_OK;
    cudaStreamSynchronize(st);
    hss_free(w);
    size_t want = bytes + bytes / 4;
    if (cudaMalloc(&w.base, want) != cudaSuccess) {
        cudaGetLastError();
        return TDEIG_ENOMEM;
    }
    w.cap = want;
    return TDEIG_OK;
}

#define HCU(x)                                                                         \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess) {                                                       \
            fprintf(stderr, "tdeig hss: %s (%s:%d)\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
            return TDEIG_ECUDA;                                                        \
        }                                                                              \
    } while (0)

// ADC1: HSS generators U, V (and the skeleton indices) level by level by SRRSC;
// D and B come from the generators as in Algorithm 2.
// The ranks of tree level l of every merge, one copy (the level's nodes hold
// consecutive rank pairs), then a synchronisation.
static int read_level_ranks(std::vector<HMerge>& H, int l, cudaStream_t st)
{
    const int* base = nullptr;
    size_t cnt = 0;
    for (auto& h : H) {
        if (l > h.L) continue;
        if (!base) base = h.nodes[hidx(l, 0)].rk;
        cnt += (size_t)1 << l;
    }
    if (!base) return TDEIG_OK;
    static thread_local std::vector<int> buf;
    buf.resize(2 * cnt);
    HCU(cudaMemcpyAsync(buf.data(), base, 2 * cnt * sizeof(int), cudaMemcpyDeviceToHost, st));
    HCU(cudaStreamSynchronize(st));
    size_t i = 0;
    for (auto& h : H) {
        if (l > h.L) continue;
        for (int q = 0; q < (1 << l); q++, i++) {
            HNode& nd = h.nodes[hidx(l, q)];
            nd.kU = buf[2 * i];
            nd.kV = buf[2 * i + 1];
        }
    }
    return TDEIG_OK;
}

static int srrsc_levels(const tdeig_options& opt, std::vector<HMerge>& H, int Lmax, FillDesc* dfill,
                        SrrscDesc* dsr, char* sr_base, size_t sr_bytes, int* status, cudaStream_t st)
{
    for (int l = Lmax; l >= 1; l--) {
        std::vector<FillDesc> fills;
        std::vector<SrrscDesc> sd;
        Bump S{sr_base, 0, sr_bytes};
        for (auto& h : H) {
            if (l > h.L) continue;
            const int s = h.s, w = 1 << (h.L - l);
            FillDesc f;
            memset(&f, 0, sizeof(f));
            f.d = h.d; f.gam = h.gam; f.mu = h.mu; f.uhat = h.uh; f.v = h.v;
            for (int q = 0; q < (1 << l); q++) {
                HNode& nd = h.nodes[hidx(l, q)];
                const int s0 = h.bounds[q * w], s1 = h.bounds[(q + 1) * w];
                const int nc = h.K - (s1 - s0);
                SrrscDesc a;
                memset(&a, 0, sizeof(a));
                a.K = h.K; a.s0 = s0; a.s1 = s1; a.kcap = s; a.ldu = nd.ldU;
                a.d = h.d; a.gam = h.gam; a.mu = h.mu; a.uh = h.uh; a.v = h.v;
                HNode* c1 = nullptr;
                HNode* c2 = nullptr;
                if (l == h.L) {
                    f.out = nd.D; f.ld = h.mcap; f.nr = f.nc = s1 - s0; f.r0 = f.c0 = s0;
                    f.rows = f.cols = nullptr;
                    fills.push_back(f);
                    a.m = s1 - s0; a.base = s0;
                } else {
                    c1 = &h.nodes[hidx(l + 1, 2 * q)];
                    c2 = &h.nodes[hidx(l + 1, 2 * q + 1)];
                    f.ld = s; f.r0 = f.c0 = 0;
                    f.out = c1->B; f.rows = c1->I; f.nr = c1->kU; f.cols = c2->J; f.nc = c2->kV;
                    fills.push_back(f);
                    f.out = c2->B; f.rows = c2->I; f.nr = c2->kU; f.cols = c1->J; f.nc = c1->kV;
                    fills.push_back(f);
                }
                for (int side = 0; side < 2; side++) {
                    SrrscDesc b = a;
                    b.side = side;
                    if (c1) {
                        b.map1 = side ? c1->J : c1->I;
                        b.n1 = side ? c1->kV : c1->kU;
                        b.map2 = side ? c2->J : c2->I;
                        b.m = b.n1 + (side ? c2->kV : c2->kU);
                    }
                    b.invd = S.take<float>((size_t)8 * nc);   // the columns' pole data
                    b.g = S.take<double>(b.m);
                    b.h = S.take<double>(nc);
                    b.gf = S.take<float>(b.m);
                    b.hf = S.take<float>(nc);
                    b.actr = S.take<unsigned char>(b.m);
                    b.actc = S.take<unsigned char>(nc);
                    b.mult = S.take<double>((size_t)b.m * s);
                    b.U = side ? nd.V : nd.U;
                    b.out_idx = side ? nd.J : nd.I;
                    b.out_piv = side ? nd.pivJ : nd.pivI;
                    b.out_rank = nd.rk + side;
                    sd.push_back(b);
                }
            }
        }
        if (S.off > S.cap || sd.size() > 8192) return TDEIG_ENOMEM;
        launch_fill(fills, dfill, st);
        HCU(cudaMemcpyAsync(dsr, sd.data(), sd.size() * sizeof(SrrscDesc), cudaMemcpyHostToDevice, st));
        td_prof_begin(st);
        k_srrsc<<<(unsigned)sd.size(), SR_NT, 0, st>>>(dsr, opt.tol, status);
        td_prof_end(st, "k_srrsc");
        HCU(cudaGetLastError());
        const int rr = read_level_ranks(H, l, st);
        if (rr) return rr;
    }
    return TDEIG_OK;
}

static int leaf_levels(int K, int m)
{
    if (K < 2 * m) return K >= 2 ? 1 : 0;
    int L = (int)lround(log2((double)K / m));
    return std::max(1, L);
}

// An ID that stopped at the sample size s with more than s rows: its rank is
// only a lower bound and the sampled residual of the node is not certified.
static bool node_saturated(const HMerge& h, int l, int q)
{
    const HNode& nd = h.nodes[hidx(l, q)];
    int mu, mv;
    if (l == h.L) {
        mu = mv = nd.r1 - nd.r0;
    } else {
        const HNode& c1 = h.nodes[hidx(l + 1, 2 * q)];
        const HNode& c2 = h.nodes[hidx(l + 1, 2 * q + 1)];
        mu = c1.kU + c2.kU;
        mv = c1.kV + c2.kV;
    }
    return (nd.kU >= h.s && mu > h.s) || (nd.kV >= h.s && mv > h.s);
}

int hss_update_level(const tdeig_options& opt, int variant, int prec,
                     const std::vector<MergeDesc>& merges, const MergeDesc* dev_merges,
                     const std::vector<int>& Kv, const LevelWS& lws, HssWS& hws, int* status,
                     cudaStream_t st, std::string& js,
                     const std::function<int(const char*)>& mark, SplitWS* split,
                     HssLearn* learn)
{
    int prc = TDEIG_OK;
    const int split_kind = prec == TDEIG_PREC_BF16X2 ? SPLIT_BF16X2
                           : prec == TDEIG_PREC_FP16X2 ? SPLIT_FP16X2 : SPLIT_OZAKI;
    auto run = [&](const std::vector<GemmDesc>& gv, GemmDesc* dev) -> double {
        if (!split) return hss_launch_gemm(gv, dev, st);
        int r = TDEIG_OK;
        double f = split_launch_gemm(gv, *split, st, &r, status, split_kind, TD_SPLIT_BITS);
        if (r && !prc) prc = r;
        return f;
    };
    double fl_dense = 0.0, fl_sample = 0.0, fl_sample_split = 0.0, fl_build = 0.0, fl_mult = 0.0;
    (void)dev_merges;
    const int p_over = opt.oversample;
    std::vector<HMerge> H;
    std::vector<GemmDesc> dense;   // merges of this level that stay dense
    for (size_t i = 0; i < merges.size(); i++) {
        const MergeDesc& md = merges[i];
        const int K = Kv[i];
        if (K == 0) continue;
        const int g0 = md.g0;
        const int L = leaf_levels(K, opt.hss_leaf);
        const int mcap_guess = (K + (1 << L) - 1) / (1 << L) + 2 * opt.boundary_shift + 2;
        const int s_max = opt.rank_cap + p_over;
        const bool fits =
            L >= 1 && (variant == TDEIG_MODE_ADC1
                           ? mcap_guess <= SR_MAXM
                           : id_smem(s_max, std::max(mcap_guess, 2 * s_max)) <= 220 * 1024);
        if (K <= opt.hss_threshold || !fits) {
            GemmDesc g;
            memset(&g, 0, sizeof(g));
            g.A = md.W; g.lda = md.n; g.acol = lws.survIdx + g0;
            g.B = md.qhat; g.ldb = K;
            g.C = md.qout; g.ldc = md.n; g.ccol = lws.posNew + g0;
            g.M = md.n; g.N = K; g.Kd = K; g.alpha = 1.0; g.beta = 0.0;
            dense.push_back(g);
            continue;
        }
        HMerge h;
        h.mi = (int)i; h.K = K; h.n = md.n; h.L = L;
        h.node_id = md.node_id;
        h.bounds.resize((1 << L) + 1);
        for (int q = 0; q <= (1 << L); q++) h.bounds[q] = (int)(((int64_t)q * K) >> L);
        h.d = lws.dK + g0; h.gam = lws.gamK + g0; h.mu = lws.muK + g0;
        h.uh = lws.uhat + g0; h.v = lws.vv + g0; h.qhat = md.qhat;
        h.surv = lws.survIdx + g0; h.posNew = lws.posNew + g0;
        h.W = md.W; h.qout = md.qout;
        H.push_back(h);
    }

    // small scratch for descriptors, bounds, ranks
    size_t desc_bytes = 1 << 20;
    for (auto& h : H) desc_bytes += ((1 << h.L) + 8) * 64 * 4;
    const bool adc2 = (variant == TDEIG_MODE_ADC2);
    const bool want_feat = learn && adc2 && (learn->record || (learn->seed && learn->model));
    size_t nfeat = 0;   // HSS nodes (all levels) of all merges
    for (auto& h : H) { h.feat0 = nfeat; nfeat += ((size_t)2 << h.L) - 2; }
    const size_t feat_bytes =
        want_feat ? nfeat * (sizeof(NodeFeatDesc) + (MLP_IN + 1) * sizeof(float)) + 4096 : 0;
    int rc = grow(hws, 4096 * sizeof(GemmDesc) + desc_bytes + feat_bytes + 64 * 1024, st);
    if (rc) return rc;
    Bump b0{hws.base, 0, hws.cap};
    GemmDesc* dgemm = b0.take<GemmDesc>(4096);
    if (!dense.empty()) fl_dense += run(dense, dgemm);
    if (H.empty()) return TDEIG_OK;
    const bool adc1 = (variant == TDEIG_MODE_ADC1);

    // ---- rank estimate and boundary moves (ADC2) -------------------------
    if (adc1) {
        // no sampling: the generator columns only bound the ranks SRRSC may reach
        for (auto& h : H) h.r = std::min(opt.rank_cap, SR_MAXK - p_over);
    } else {
        std::vector<RankDesc> rd;
        int* ib = b0.take<int>(desc_bytes / 8);
        size_t o = 0;
        for (auto& h : H) {
            h.dev_bounds = ib + o; o += h.bounds.size();
            h.dev_r = ib + o; o += 1;
            HCU(cudaMemcpyAsync(h.dev_bounds, h.bounds.data(), h.bounds.size() * sizeof(int),
                                cudaMemcpyHostToDevice, st));
            RankDesc r;
            r.d = h.d; r.gam = h.gam; r.K = h.K; r.nl = 1 << h.L;
            r.bounds = h.dev_bounds; r.r_out = h.dev_r;
            rd.push_back(r);
        }
        RankDesc* drd = b0.take<RankDesc>(rd.size());
        HCU(cudaMemcpyAsync(drd, rd.data(), rd.size() * sizeof(RankDesc), cudaMemcpyHostToDevice, st));
        td_prof_begin(st);
        k_rank_estimate<<<td_cdiv((int)rd.size(), 64), 64, 0, st>>>(drd, (int)rd.size(), opt.rank_eps,
                                                                   opt.rank_cap, opt.boundary_shift);
        td_prof_end(st, "k_rank_estimate");
        for (auto& h : H) {
            HCU(cudaMemcpyAsync(h.bounds.data(), h.dev_bounds, h.bounds.size() * sizeof(int),
                                cudaMemcpyDeviceToHost, st));
            HCU(cudaMemcpyAsync(&h.r, h.dev_r, sizeof(int), cudaMemcpyDeviceToHost, st));
        }
        HCU(cudaStreamSynchronize(st));
        for (auto& h : H) h.r_est = h.r;
    }

    // ---- node features and the learned seed (ADC2) ------------------------
    std::vector<float> feat_h;
    if (want_feat) {
        std::vector<NodeFeatDesc> fd;
        fd.reserve(nfeat);
        NodeFeatDesc* dfd = b0.take<NodeFeatDesc>(nfeat);
        float* dX = b0.take<float>(nfeat * MLP_IN);
        float* dy = b0.take<float>(nfeat);
        if (b0.off > b0.cap) return TDEIG_ENOMEM;
        for (auto& h : H)
            for (int l = 1; l <= h.L; l++) {
                const int w = 1 << (h.L - l);
                for (int q = 0; q < (1 << l); q++) {
                    NodeFeatDesc f;
                    f.d = h.d; f.gam = h.gam; f.mu = h.mu; f.uh = h.uh;
                    f.K = h.K; f.n = h.n;
                    f.s0 = h.bounds[q * w]; f.s1 = h.bounds[(q + 1) * w];
                    f.out = dX + (h.feat0 + hidx(l, q) - 1) * MLP_IN;
                    fd.push_back(f);
                }
            }
        HCU(cudaMemcpyAsync(dfd, fd.data(), fd.size() * sizeof(NodeFeatDesc), cudaMemcpyHostToDevice, st));
        mlp_launch_features(dfd, (int)fd.size(), st);
        std::vector<float> yh;
        if (learn->seed && learn->model) {
            mlp_launch(learn->model, learn->model + MLP_P, learn->model + MLP_P + MLP_IN, dX, nullptr,
                       nullptr, (int)nfeat, (int)nfeat, dy, nullptr, nullptr, st);
            yh.resize(nfeat);
            HCU(cudaMemcpyAsync(yh.data(), dy, nfeat * sizeof(float), cudaMemcpyDeviceToHost, st));
        }
        if (learn->record) {
            feat_h.resize(nfeat * MLP_IN);
            HCU(cudaMemcpyAsync(feat_h.data(), dX, nfeat * MLP_IN * sizeof(float), cudaMemcpyDeviceToHost, st));
        }
        HCU(cudaStreamSynchronize(st));
        HCU(cudaGetLastError());
        if (!yh.empty()) {
            // r = ceil(exp(max over the merge's nodes of the predicted ln(rank + 1)) - 1)
            for (auto& h : H) {
                float ymax = -1e30f;
                for (size_t i = h.feat0; i < h.feat0 + ((size_t)2 << h.L) - 2; i++) ymax = fmaxf(ymax, yh[i]);
                const double rr = ceil(exp(std::min((double)ymax, 10.0)) - 1.0);
                h.r = (int)std::max(1.0, std::min((double)opt.rank_cap, rr));
                h.seed = 1;
            }
        }
    }

    // A merge seeded by the model is accepted unless one of its IDs reached the
    // sample size with more rows than that (its sampled residual is then not
    // certified); such a merge is rebuilt with the estimate when the estimate
    // samples more, else kept (the estimate would have reached the same bound).
    Bump B{hws.base, 0, hws.cap};
    FillDesc* dfill = nullptr;
    IdDesc* did = nullptr;
    GatherDesc* dgat = nullptr;
    int Lmax = 0;
    for (int attempt = 0;; attempt++) {
    // ---- sizes and allocation ---------------------------------------------
    size_t total = b0.off + 1024;
    for (auto& h : H) {
        h.s = h.r + p_over;
        int mc = 0;
        for (int q = 0; q < (1 << h.L); q++) mc = std::max(mc, h.bounds[q + 1] - h.bounds[q]);
        h.mcap = mc;
        const size_t s = h.s, nl = (size_t)1 << h.L, K = h.K, n = h.n, two_s = 2 * s;
        total += 3 * K * s * 8 + K * 4 + 256;                  // Om, Y, Z, leaf_of
        total += nl * (2 * mc * s + (size_t)mc * mc) * 8;       // leaves U, V, D
        total += 2 * nl * (4 * two_s * s) * 8;                 // parents Phi, Theta, U, V, Ystk, Zstk
        total += 2 * nl * (s * s) * 8;                         // B
        total += 2 * nl * (4 * s + 2) * 4;                     // I, J, piv, rk
        for (int l = 1; l <= h.L; l++) total += 2 * n * (((size_t)1 << l) * s) * 8;  // G, F
        total += 2 * nl * 8 * 256;                             // alignment slack
    }
    size_t sr_bytes = 0;   // ADC1 elimination scratch, reused level by level
    if (adc1) {
        for (auto& h : H) {
            const size_t nl = (size_t)1 << h.L, K = h.K, mc = std::max(h.mcap, 2 * h.s);
            sr_bytes += 2 * nl * (mc * K * 4 + (mc + K) * 14 + mc * h.s * 8 + 8 * 256);
        }
        total += sr_bytes + 2 * 8192 * sizeof(SrrscDesc);
    }
    if (total > hws.cap) {
        // keep the small region (bounds already read back) and regrow
        rc = grow(hws, total, st);
        if (rc) return rc;
        b0 = Bump{hws.base, 0, hws.cap};
        dgemm = b0.take<GemmDesc>(4096);
        b0.take<int>(desc_bytes / 8);
    }
    B = Bump{hws.base, b0.off, hws.cap};
    dfill = B.take<FillDesc>(8192);
    did = B.take<IdDesc>(8192);
    dgat = B.take<GatherDesc>(8192);
    for (auto& h : H) {
        const int s = h.s, K = h.K, nn = h.n;
        h.Om = B.take<double>((size_t)K * s);
        h.Y = B.take<double>((size_t)K * s);
        h.Z = B.take<double>((size_t)K * s);
        h.leaf_of = B.take<int>((size_t)K);
        h.nodes.assign((size_t)2 << h.L, HNode());
        for (int l = 1; l <= h.L; l++) {
            for (int q = 0; q < (1 << l); q++) {
                HNode& nd = h.nodes[hidx(l, q)];
                nd.I = B.take<int>(s); nd.J = B.take<int>(s);
                nd.pivI = B.take<int>(s); nd.pivJ = B.take<int>(s);
                nd.B = B.take<double>((size_t)s * s);
                if (l == h.L) {
                    nd.r0 = h.bounds[q]; nd.r1 = h.bounds[q + 1];
                    nd.ldU = h.mcap;
                    nd.U = B.take<double>((size_t)h.mcap * s);
                    nd.V = B.take<double>((size_t)h.mcap * s);
                    nd.D = B.take<double>((size_t)h.mcap * h.mcap);
                    nd.Phi = h.Y + nd.r0; nd.Theta = h.Z + nd.r0; nd.ldPhi = K;
                } else {
                    nd.ldU = 2 * s;
                    nd.U = B.take<double>((size_t)2 * s * s);
                    nd.V = B.take<double>((size_t)2 * s * s);
                    nd.Phi = B.take<double>((size_t)2 * s * s);
                    nd.Theta = B.take<double>((size_t)2 * s * s);
                    nd.ldPhi = 2 * s;
                    nd.Ystk = B.take<double>((size_t)2 * s * s);
                    nd.Zstk = B.take<double>((size_t)2 * s * s);
                }
            }
        }
        h.G.assign(h.L + 1, nullptr);
        h.F.assign(h.L + 1, nullptr);
        for (int l = 1; l <= h.L; l++) {
            h.G[l] = B.take<double>((size_t)nn * ((size_t)1 << l) * s);
            h.F[l] = B.take<double>((size_t)nn * ((size_t)1 << l) * s);
        }
    }
    {
        // ranks (kU, kV) of every node, level by level, so that one copy per
        // tree level brings a level's ranks to the host
        size_t total = 0;
        int lm = 0;
        for (auto& h : H) {
            lm = std::max(lm, h.L);
            for (int l = 1; l <= h.L; l++) total += (size_t)1 << l;
        }
        int* rk_all = B.take<int>(2 * std::max<size_t>(total, 1));
        size_t idx = 0;
        for (int l = 1; l <= lm; l++)
            for (auto& h : H) {
                if (l > h.L) continue;
                for (int q = 0; q < (1 << l); q++) h.nodes[hidx(l, q)].rk = rk_all + 2 * idx++;
            }
    }
    SrrscDesc* dsr = nullptr;
    char* sr_base = nullptr;
    if (adc1) {
        dsr = B.take<SrrscDesc>(8192);
        sr_base = B.take<char>(sr_bytes);
    }
    if (B.off > B.cap) return TDEIG_ENOMEM;

    Lmax = 0;
    for (auto& h : H) Lmax = std::max(Lmax, h.L);
    if (adc1) {
        if ((rc = mark("hss_build"))) return rc;
        rc = srrsc_levels(opt, H, Lmax, dfill, dsr, sr_base, sr_bytes, status, st);
        if (rc) return rc;
    }

    if (!adc1 && (rc = mark("hss_sample"))) return rc;
    // ---- sampling: Omega, Y = A Omega, Z = A^T Omega (Omega(1) = Omega(2)) --
    // Split sampling multiplies the off-diagonal part of Qhat (the leaf blocks
    // masked to zero), which is Phi / Theta of the leaves directly.  A split
    // product of the whole Qhat carries errors relative to the row and column
    // maxima (the large near-diagonal entries), far above the small
    // off-diagonal entries that Phi = Y - D Omega keeps after the cancellation.
    const bool masked = split && prec == TDEIG_PREC_SPLIT && !adc1;
    std::vector<std::vector<int>> leaf_ids;
    if (masked) {
        for (auto& h : H) {
            leaf_ids.emplace_back(h.K);
            std::vector<int>& v = leaf_ids.back();
            for (int q = 0; q < (1 << h.L); q++)
                for (int i = h.bounds[q]; i < h.bounds[q + 1]; i++) v[i] = q;
            HCU(cudaMemcpyAsync(h.leaf_of, v.data(), h.K * sizeof(int), cudaMemcpyHostToDevice, st));
        }
    }
    std::vector<GemmDesc> gl;
    for (auto& h : H) {
        if (adc1) break;
        const int64_t tot = (int64_t)h.K * h.s;
        td_prof_begin(st);
        k_philox_omega<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(h.Om, h.K, h.s, opt.seed,
                                                                      (unsigned)h.node_id);
        td_prof_end(st, "k_philox_omega");
        GemmDesc g;
        memset(&g, 0, sizeof(g));
        g.A = h.qhat; g.lda = h.K; g.B = h.Om; g.ldb = h.K; g.C = h.Y; g.ldc = h.K;
        g.M = h.K; g.N = h.s; g.Kd = h.K; g.alpha = 1.0;
        g.amask = masked ? h.leaf_of : nullptr;
        gl.push_back(g);
        g.transA = 1; g.C = h.Z;
        gl.push_back(g);
    }
    // Split sampling keeps 56 bits (products as accurate as FP64 ones); the
    // two-slice variants sample in FP64.
    if (masked) {
        int r = TDEIG_OK;
        fl_sample_split += split_launch_gemm(gl, *split, st, &r, status, SPLIT_OZAKI, TD_SAMPLE_BITS);
        if (r) return r;
    } else {
        fl_sample += hss_launch_gemm(gl, dgemm, st);
    }

    if (!adc1 && (rc = mark("hss_build"))) return rc;
    // ---- Algorithm 2, levels L..1 -------------------------------------------
    for (int l = adc1 ? 0 : Lmax; l >= 1; l--) {
        std::vector<FillDesc> fills;
        std::vector<GatherDesc> gathers;
        std::vector<GemmDesc> upd;
        std::vector<IdDesc> ids;
        for (auto& h : H) {
            if (l > h.L) continue;
            const int s = h.s;
            for (int q = 0; q < (1 << l); q++) {
                HNode& nd = h.nodes[hidx(l, q)];
                if (l == h.L) {
                    const int m = nd.r1 - nd.r0;
                    FillDesc f;
                    memset(&f, 0, sizeof(f));
                    f.out = nd.D; f.ld = h.mcap; f.nr = m; f.nc = m; f.r0 = nd.r0; f.c0 = nd.r0;
                    f.d = h.d; f.gam = h.gam; f.mu = h.mu; f.uhat = h.uh; f.v = h.v;
                    fills.push_back(f);
                    if (!masked) {   // masked sampling produced Phi_i, Theta_i directly
                        GemmDesc g;
                        memset(&g, 0, sizeof(g));
                        g.A = nd.D; g.lda = h.mcap; g.B = h.Om + nd.r0; g.ldb = h.K;
                        g.C = nd.Phi; g.ldc = h.K; g.M = m; g.N = s; g.Kd = m;
                        g.alpha = -1.0; g.beta = 1.0;
                        upd.push_back(g);            // Phi_i = Y_i - D_i Omega_i
                        g.transA = 1; g.C = nd.Theta;
                        upd.push_back(g);            // Theta_i = Z_i - D_i^T Omega_i
                    }
                    IdDesc a;
                    memset(&a, 0, sizeof(a));
                    a.Phi = nd.Phi; a.ldphi = h.K; a.m = m; a.s = s; a.rowbase = nd.r0;
                    a.U = nd.U; a.ldu = nd.ldU; a.out_idx = nd.I; a.out_piv = nd.pivI; a.out_rank = nd.rk;
                    ids.push_back(a);
                    a.Phi = nd.Theta; a.U = nd.V; a.out_idx = nd.J; a.out_piv = nd.pivJ; a.out_rank = nd.rk + 1;
                    ids.push_back(a);
                } else {
                    HNode& c1 = h.nodes[hidx(l + 1, 2 * q)];
                    HNode& c2 = h.nodes[hidx(l + 1, 2 * q + 1)];
                    FillDesc f;
                    memset(&f, 0, sizeof(f));
                    f.d = h.d; f.gam = h.gam; f.mu = h.mu; f.uhat = h.uh; f.v = h.v; f.ld = s;
                    f.out = c1.B; f.rows = c1.I; f.nr = c1.kU; f.cols = c2.J; f.nc = c2.kV;
                    fills.push_back(f);           // B_{c1} = A(I_{c1}, J_{c2})
                    f.out = c2.B; f.rows = c2.I; f.nr = c2.kU; f.cols = c1.J; f.nc = c1.kV;
                    fills.push_back(f);           // B_{c2} = A(I_{c2}, J_{c1})
                    GatherDesc gd;
                    gd.ncols = s; gd.ldd = 2 * s;
                    gd.src = c1.Phi; gd.lds = c1.ldPhi; gd.piv = c1.pivI; gd.nr = c1.kU; gd.dst = nd.Phi;
                    gathers.push_back(gd);
                    gd.src = c2.Phi; gd.lds = c2.ldPhi; gd.piv = c2.pivI; gd.nr = c2.kU; gd.dst = nd.Phi + c1.kU;
                    gathers.push_back(gd);
                    gd.src = c1.Theta; gd.lds = c1.ldPhi; gd.piv = c1.pivJ; gd.nr = c1.kV; gd.dst = nd.Theta;
                    gathers.push_back(gd);
                    gd.src = c2.Theta; gd.lds = c2.ldPhi; gd.piv = c2.pivJ; gd.nr = c2.kV; gd.dst = nd.Theta + c1.kV;
                    gathers.push_back(gd);
                    GemmDesc g;
                    memset(&g, 0, sizeof(g));
                    g.alpha = -1.0; g.beta = 1.0; g.ldc = 2 * s; g.N = s; g.ldb = 2 * s; g.lda = s;
                    // Phi rows of c1 -= B_{c1} Yhat_{c2}
                    g.A = c1.B; g.M = c1.kU; g.Kd = c2.kV; g.B = nd.Ystk + c1.kV; g.C = nd.Phi;
                    upd.push_back(g);
                    // Phi rows of c2 -= B_{c2} Yhat_{c1}
                    g.A = c2.B; g.M = c2.kU; g.Kd = c1.kV; g.B = nd.Ystk; g.C = nd.Phi + c1.kU;
                    upd.push_back(g);
                    // Theta rows of c1 -= B_{c2}^T Zhat_{c2}
                    g.transA = 1;
                    g.A = c2.B; g.M = c1.kV; g.Kd = c2.kU; g.B = nd.Zstk + c1.kU; g.C = nd.Theta;
                    upd.push_back(g);
                    // Theta rows of c2 -= B_{c1}^T Zhat_{c1}
                    g.A = c1.B; g.M = c2.kV; g.Kd = c1.kU; g.B = nd.Zstk; g.C = nd.Theta + c1.kV;
                    upd.push_back(g);
                    IdDesc a;
                    memset(&a, 0, sizeof(a));
                    a.Phi = nd.Phi; a.ldphi = 2 * s; a.m = c1.kU + c2.kU; a.s = s;
                    a.U = nd.U; a.ldu = 2 * s; a.out_idx = nd.I; a.out_piv = nd.pivI; a.out_rank = nd.rk;
                    // stacked rows: the children's skeleton rows, c1's then c2's
                    a.rowmap = c1.I; a.rowmap2 = c2.I; a.n1 = c1.kU;
                    ids.push_back(a);
                    a.Phi = nd.Theta; a.m = c1.kV + c2.kV; a.U = nd.V; a.out_idx = nd.J;
                    a.out_piv = nd.pivJ; a.out_rank = nd.rk + 1;
                    a.rowmap = c1.J; a.rowmap2 = c2.J; a.n1 = c1.kV;
                    ids.push_back(a);
                }
            }
        }
        launch_fill(fills, dfill, st);
        launch_gather(gathers, dgat, st);
        fl_build += hss_launch_gemm(upd, dgemm, st);
        if (!ids.empty()) {
            HCU(cudaMemcpyAsync(did, ids.data(), ids.size() * sizeof(IdDesc), cudaMemcpyHostToDevice, st));
            int mmax = 0, smax = 0;
            for (auto& a : ids) { mmax = std::max(mmax, a.m); smax = std::max(smax, a.s); }
            size_t sm = id_smem(smax, mmax);
            td_smem_attr((const void*)k_id, 220 * 1024);
            td_prof_begin(st);
            k_id<<<(unsigned)ids.size(), HSS_NT, sm, st>>>(did, (int)ids.size(), opt.tol);
            td_prof_end(st, "k_id");
            HCU(cudaGetLastError());
        }
        // ranks back to the host
        if ((rc = read_level_ranks(H, l, st))) return rc;
        // Yhat_i = V_i^T (Omega_i or stacked children Yhat), Zhat_i = U_i^T (...),
        // stacked into the parent (levels >= 2 only: the root needs no Phi).
        if (l >= 2) {
            std::vector<GemmDesc> yz;
            for (auto& h : H) {
                if (l > h.L) continue;
                const int s = h.s;
                for (int q = 0; q < (1 << l); q++) {
                    HNode& nd = h.nodes[hidx(l, q)];
                    HNode& par = h.nodes[hidx(l - 1, q >> 1)];
                    HNode& left = h.nodes[hidx(l, q & ~1)];
                    const int offV = (q & 1) ? left.kV : 0, offU = (q & 1) ? left.kU : 0;
                    GemmDesc g;
                    memset(&g, 0, sizeof(g));
                    g.transA = 1; g.alpha = 1.0; g.N = s; g.ldc = 2 * s;
                    if (l == h.L) {
                        const int m = nd.r1 - nd.r0;
                        g.A = nd.V; g.lda = nd.ldU; g.M = nd.kV; g.Kd = m;
                        g.B = h.Om + nd.r0; g.ldb = h.K; g.C = par.Ystk + offV;
                        yz.push_back(g);
                        g.A = nd.U; g.M = nd.kU; g.C = par.Zstk + offU;
                        yz.push_back(g);
                    } else {
                        HNode& c1 = h.nodes[hidx(l + 1, 2 * q)];
                        HNode& c2 = h.nodes[hidx(l + 1, 2 * q + 1)];
                        g.A = nd.V; g.lda = 2 * s; g.M = nd.kV; g.Kd = c1.kV + c2.kV;
                        g.B = nd.Ystk; g.ldb = 2 * s; g.C = par.Ystk + offV;
                        yz.push_back(g);
                        g.A = nd.U; g.M = nd.kU; g.Kd = c1.kU + c2.kU; g.B = nd.Zstk; g.C = par.Zstk + offU;
                        yz.push_back(g);
                    }
                }
            }
            fl_build += hss_launch_gemm(yz, dgemm, st);
        }
    }
    // root: B of its two children
    {
        std::vector<FillDesc> fills;
        for (auto& h : H) {
            HNode& c1 = h.nodes[hidx(1, 0)];
            HNode& c2 = h.nodes[hidx(1, 1)];
            FillDesc f;
            memset(&f, 0, sizeof(f));
            f.d = h.d; f.gam = h.gam; f.mu = h.mu; f.uhat = h.uh; f.v = h.v; f.ld = h.s;
            f.out = c1.B; f.rows = c1.I; f.nr = c1.kU; f.cols = c2.J; f.nc = c2.kV;
            fills.push_back(f);
            f.out = c2.B; f.rows = c2.I; f.nr = c2.kU; f.cols = c1.J; f.nc = c1.kV;
            fills.push_back(f);
        }
        launch_fill(fills, dfill, st);
    }
    bool again = false;
    for (auto& h : H) {
        if (h.seed != 1 || adc1) continue;
        bool sat = false;
        for (int l = 1; l <= h.L; l++)
            for (int q = 0; q < (1 << l); q++) sat |= node_saturated(h, l, q);
        if (sat && h.r_est > h.r) {
            h.r = h.r_est;
            h.seed = 2;
            again = true;
            if (learn) learn->fallbacks++;
        }
    }
    if (!again) break;
    }   // attempts

    if (learn && learn->record && adc2 && !feat_h.empty()) {
        // features and ln(rank + 1) of every node whose rank the IDs certified
        for (auto& h : H)
            for (int l = 1; l <= h.L; l++)
                for (int q = 0; q < (1 << l); q++) {
                    if (node_saturated(h, l, q)) continue;
                    const HNode& nd = h.nodes[hidx(l, q)];
                    const float* f = feat_h.data() + (h.feat0 + hidx(l, q) - 1) * MLP_IN;
                    learn->records->insert(learn->records->end(), f, f + MLP_IN);
                    learn->records->push_back((float)log((double)std::max(nd.kU, nd.kV) + 1.0));
                }
    }

    if ((rc = mark("hss_mult"))) return rc;
    // ---- Algorithm 3: X H with X = W[:, surv] (n x K) ----------------------
    auto colU = [](HMerge& h, int l, int q) {
        int base = (q >> 1) * 2 * h.s;
        return (q & 1) ? base + h.nodes[hidx(l, q - 1)].kU : base;
    };
    auto colV = [](HMerge& h, int l, int q) {
        int base = (q >> 1) * 2 * h.s;
        return (q & 1) ? base + h.nodes[hidx(l, q - 1)].kV : base;
    };
    {
        // upsweep: leaves G_i = X_i U_i
        std::vector<GemmDesc> g1;
        for (auto& h : H) {
            for (int q = 0; q < (1 << h.L); q++) {
                HNode& nd = h.nodes[hidx(h.L, q)];
                GemmDesc g;
                memset(&g, 0, sizeof(g));
                g.A = h.W; g.lda = h.n; g.acol = h.surv + nd.r0;
                g.B = nd.U; g.ldb = nd.ldU;
                g.C = h.G[h.L] + (size_t)colU(h, h.L, q) * h.n; g.ldc = h.n;
                g.M = h.n; g.N = nd.kU; g.Kd = nd.r1 - nd.r0; g.alpha = 1.0;
                g1.push_back(g);
            }
        }
        fl_mult += run(g1, dgemm);
        for (int l = Lmax - 1; l >= 1; l--) {
            std::vector<GemmDesc> gu;
            for (auto& h : H) {
                if (l >= h.L) continue;
                for (int q = 0; q < (1 << l); q++) {
                    HNode& nd = h.nodes[hidx(l, q)];
                    HNode& c1 = h.nodes[hidx(l + 1, 2 * q)];
                    HNode& c2 = h.nodes[hidx(l + 1, 2 * q + 1)];
                    GemmDesc g;
                    memset(&g, 0, sizeof(g));
                    g.A = h.G[l + 1] + (size_t)(2 * q * h.s) * h.n; g.lda = h.n;
                    g.B = nd.U; g.ldb = 2 * h.s;
                    g.C = h.G[l] + (size_t)colU(h, l, q) * h.n; g.ldc = h.n;
                    g.M = h.n; g.N = nd.kU; g.Kd = c1.kU + c2.kU; g.alpha = 1.0;
                    gu.push_back(g);
                }
            }
            fl_mult += run(gu, dgemm);
        }
        // downsweep
        for (int l = 1; l <= Lmax; l++) {
            std::vector<GemmDesc> gf, gv;
            for (auto& h : H) {
                if (l > h.L) continue;
                for (int q = 0; q < (1 << l); q++) {
                    HNode& nd = h.nodes[hidx(l, q)];
                    HNode& sib = h.nodes[hidx(l, q ^ 1)];
                    double* Fi = h.F[l] + (size_t)colV(h, l, q) * h.n;
                    GemmDesc g;
                    memset(&g, 0, sizeof(g));
                    g.A = h.G[l] + (size_t)colU(h, l, q ^ 1) * h.n; g.lda = h.n;
                    g.B = sib.B; g.ldb = h.s;
                    g.C = Fi; g.ldc = h.n;
                    g.M = h.n; g.N = nd.kV; g.Kd = sib.kU; g.alpha = 1.0; g.beta = (l >= 2) ? 1.0 : 0.0;
                    gf.push_back(g);                       // F_i (+)= G_j B_j
                    if (l < h.L) {
                        HNode& c1 = h.nodes[hidx(l + 1, 2 * q)];
                        HNode& c2 = h.nodes[hidx(l + 1, 2 * q + 1)];
                        GemmDesc v;
                        memset(&v, 0, sizeof(v));
                        v.A = Fi; v.lda = h.n;
                        v.B = nd.V; v.ldb = 2 * h.s; v.transB = 1;
                        v.C = h.F[l + 1] + (size_t)(2 * q * h.s) * h.n; v.ldc = h.n;
                        v.M = h.n; v.N = c1.kV + c2.kV; v.Kd = nd.kV; v.alpha = 1.0;
                        gv.push_back(v);                   // [F_c1, F_c2] = F_i V_i^T
                    }
                }
            }
            fl_mult += run(gf, dgemm);
            fl_mult += run(gv, dgemm);
        }
        // leaves: out[:, t_i] = X_i D_i + F_i V_i^T (columns scattered to their final
        // positions).  Split products take both terms in one product with two terms
        // along k (one pass over the output; X_i and F_i rows, D_i columns and V_i
        // rows are of like magnitude, so a shared exponent per row / column costs
        // little).  The same fusion in the downsweep, F_c = F_p V_p^T + G_j B_j, was
        // measured (CPU emulation of the digit products) to lose an order of
        // magnitude: there the two terms' scales differ by up to 2^14.
        std::vector<GemmDesc> gd, gvv;
        for (auto& h : H) {
            for (int q = 0; q < (1 << h.L); q++) {
                HNode& nd = h.nodes[hidx(h.L, q)];
                const int m = nd.r1 - nd.r0;
                GemmDesc g;
                memset(&g, 0, sizeof(g));
                g.A = h.W; g.lda = h.n; g.acol = h.surv + nd.r0;
                g.B = nd.D; g.ldb = h.mcap;
                g.C = h.qout; g.ldc = h.n; g.ccol = h.posNew + nd.r0;
                g.M = h.n; g.N = m; g.Kd = m; g.alpha = 1.0;
                GemmDesc v;
                memset(&v, 0, sizeof(v));
                v.A = h.F[h.L] + (size_t)colV(h, h.L, q) * h.n; v.lda = h.n;
                v.B = nd.V; v.ldb = nd.ldU; v.transB = 1;
                v.C = h.qout; v.ldc = h.n; v.ccol = h.posNew + nd.r0;
                v.M = h.n; v.N = m; v.Kd = nd.kV; v.alpha = 1.0; v.beta = 1.0;
                if (split) {
                    g.A2 = v.A; g.lda2 = v.lda;
                    g.B2 = v.B; g.ldb2 = v.ldb; g.transB2 = 1;
                    g.Kd2 = v.Kd;
                    gd.push_back(g);
                } else {
                    gd.push_back(g);
                    gvv.push_back(v);
                }
            }
        }
        fl_mult += run(gd, dgemm);
        if (!gvv.empty()) fl_mult += run(gvv, dgemm);
    }
    HCU(cudaGetLastError());

    // statistics
    char buf[256];
    snprintf(buf, sizeof(buf),
             "%s{\"flops\":{\"dense\":%.6e,\"sample\":%.6e,\"sample_split\":%.6e,\"build\":%.6e,"
             "\"mult\":%.6e}}",
             js.empty() ? "" : ",", fl_dense, fl_sample, fl_sample_split, fl_build, fl_mult);
    js += buf;
    for (auto& h : H) {
        int kmax = 0;
        double ksum = 0.0;
        int cnt = 0;
        for (int l = 1; l <= h.L; l++)
            for (int q = 0; q < (1 << l); q++) {
                HNode& nd = h.nodes[hidx(l, q)];
                kmax = std::max(kmax, std::max(nd.kU, nd.kV));
                ksum += nd.kU + nd.kV;
                cnt += 2;
            }
        snprintf(buf, sizeof(buf),
                 "%s{\"n\":%d,\"K\":%d,\"L\":%d,\"r\":%d,\"s\":%d,\"kmax\":%d,\"kmean\":%.2f,"
                 "\"r_est\":%d,\"seed\":%d,\"node\":%d,\"bounds\":[",
                 js.empty() ? "" : ",", h.n, h.K, h.L, h.r, h.s, kmax, cnt ? ksum / cnt : 0.0, h.r_est,
                 h.seed, h.node_id);
        js += buf;
        // the (moved) leaf boundaries, then every node's (row, column) ID ranks,
        // levels 1..L left to right
        for (size_t q = 0; q < h.bounds.size(); q++) {
            snprintf(buf, sizeof(buf), "%s%d", q ? "," : "", h.bounds[q]);
            js += buf;
        }
        js += "],\"node_ranks\":[";
        bool first = true;
        for (int l = 1; l <= h.L; l++)
            for (int q = 0; q < (1 << l); q++) {
                const HNode& nd = h.nodes[hidx(l, q)];
                snprintf(buf, sizeof(buf), "%s[%d,%d]", first ? "" : ",", nd.kU, nd.kV);
                js += buf;
                first = false;
            }
        js += "]}";
    }
    return prc;
}
