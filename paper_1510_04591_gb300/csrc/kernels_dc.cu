// Kernels of the divide-and-conquer merge path (Algorithm 1 of Li, Liao, Liu,
// Jiang), batched over every merge of one level of the DC tree.  All
// arithmetic is IEEE FP64.
//
//   k_scale_input   scale each matrix by max(|a|, |b|)
//   k_leaf_qr       QR algorithm with Wilkinson shift on each leaf (thread per leaf), rotations recorded
//   k_leaf_apply    the rotations applied to Q (warp per leaf), eigenpairs sorted
//   k_prep          eq. T3: u from the children's Q rows; sort; deflation
//                   (tiny z and close-pole Givens tests); compaction
//   k_build_w       sorted diag(Q1, Q2) columns with the deflation rotations applied
//   k_secular       Theorem 1 roots, one warp per root, with gamma/mu of Remark 1
//   k_lowner        eq. ev_z, one warp per entry
//   k_cauchy        eq. Ev-Q column normalisation and the Cauchy-like matrix
//   k_order         merge of new and deflated eigenvalues (final ordering)
//   k_gemm_f64      dense update diag(Q1, Q2) P Qhat (plain DC)
//   k_copy_defl     deflated eigenvectors to their final columns
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>

#include "../../include/tdeig.h"
#include "common.cuh"

#define TD_NOALLOC_MAX_DEVICES 64

static thread_local TdCtx t_idle_ctx;            // counts of launches outside handle calls
static thread_local TdCtx* t_ctx = nullptr;

TdCtx& td_ctx() { return t_ctx ? *t_ctx : t_idle_ctx; }
TdCtxScope::TdCtxScope(TdCtx* c) : prev(t_ctx) { t_ctx = c; }
TdCtxScope::~TdCtxScope() { t_ctx = prev; }

#define TD_MAX_DEVICES 64
static std::mutex g_attr_mu;

void td_smem_attr(const void* kernel, size_t bytes)
{
    // per (kernel, device): the largest limit set so far
    static std::vector<std::pair<const void*, size_t>> done[TD_MAX_DEVICES];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= TD_MAX_DEVICES) {
        cudaGetLastError();
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        return;
    }
    std::lock_guard<std::mutex> lock(g_attr_mu);
    for (auto& e : done[dev])
        if (e.first == kernel) {
            if (e.second >= bytes) return;
            cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
            e.second = bytes;
            return;
        }
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    done[dev].push_back({kernel, bytes});
}

int td_sm_count()
{
    static int nsm[TD_MAX_DEVICES];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= TD_MAX_DEVICES) {
        cudaGetLastError();
        return 1;
    }
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (!nsm[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        nsm[dev] = n > 0 ? n : 1;
    }
    return nsm[dev];
}

static cudaEvent_t prof_next(TdProf& P, const char* name)
{
    if (P.n >= P.ev.size()) {
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        P.ev.push_back(e);
        P.name.push_back(nullptr);
        P.note.emplace_back();
    }
    P.name[P.n] = name;
    P.note[P.n].clear();
    return P.ev[P.n++];
}

void td_prof_begin(cudaStream_t st)
{
    TdProf& P = td_ctx().prof;
    if (P.on) cudaEventRecord(prof_next(P, nullptr), st);
}

void td_prof_note(const std::string& s)
{
    TdProf& P = td_ctx().prof;
    if (P.on && P.n > 0) P.note[P.n - 1] = s;
}

void td_prof_end(cudaStream_t st, const char* name)
{
    TdCtx& c = td_ctx();
    c.launches++;
    if (c.prof.on) cudaEventRecord(prof_next(c.prof, name), st);
}

// ---------------------------------------------------------------------------
// Input scaling: A[g] = d[g] / s_b, Bc[g] = e (row g, g+1) / s_b within member b.
// ---------------------------------------------------------------------------
// mrow0[0..members) are the first rows of the matrices, mrow0[members..2 members)
// the offsets of their off-diagonals in e.
__global__ void k_member_max(const double* d, const double* e, const int64_t* mrow0,
                             const int64_t* mN, double* scale)
{
    int b = blockIdx.x;
    int64_t r0 = mrow0[b], N = mN[b];
    const double* db = d + r0;
    const double* eb = e ? e + mrow0[gridDim.x + b] : nullptr;
    double m = 0.0;
    bool bad = false;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        double v = db[i];
        if (!isfinite(v)) bad = true;
        m = fmax(m, fabs(v));
        if (eb && i < N - 1) {
            double w = eb[i];
            if (!isfinite(w)) bad = true;
            m = fmax(m, fabs(w));
        }
    }
    __shared__ double red[32];
    __shared__ int sbad;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    if (bad) atomicOr(&sbad, 1);
    m = td_warp_max(m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
        v = td_warp_max(v);
        if (threadIdx.x == 0) scale[b] = sbad ? -1.0 : (v > 0.0 ? v : 1.0);
    }
}

__global__ void k_scale_copy(const double* d, const double* e, const int64_t* mrow0,
                             const int64_t* mN, int members, const double* scale, double* A,
                             double* Bc, int64_t R)
{
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= R) return;
    int lo = 0, hi = members - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (mrow0[mid] <= g) lo = mid; else hi = mid - 1;
    }
    int b = lo;
    double s = scale[b];
    if (s <= 0.0) s = 1.0;
    int64_t i = g - mrow0[b];
    A[g] = d[g] / s;
    Bc[g] = (e && i < mN[b] - 1) ? e[mrow0[members + b] + i] / s : 0.0;
}

void td_launch_scale_input(const double* d, const double* e, const int64_t* mrow0, const int64_t* mN,
                           int members, double* A, double* Bc, double* scale, int64_t R,
                           cudaStream_t st)
{
    td_prof_begin(st); k_member_max<<<members, 256, 0, st>>>(d, e, mrow0, mN, scale); td_prof_end(st, "k_member_max");
    if (R > 0) {
        td_prof_begin(st);
        k_scale_copy<<<(unsigned)((R + 255) / 256), 256, 0, st>>>(d, e, mrow0, mN, members, scale, A,
                                                                 Bc, R);
        td_prof_end(st, "k_scale_copy");
    }
}

// ---------------------------------------------------------------------------
// Leaf solver: symmetric tridiagonal implicit QR with Wilkinson shift
// (Algorithm 1, "use QR algorithm"), one warp per leaf of n <= 32 rows.  The
// scalar bulge chase runs redundantly in every lane (uniform control flow);
// lane r owns row r of Q, kept in shared memory.
// ---------------------------------------------------------------------------
#define LEAF_WARPS 4

// Implicit symmetric tridiagonal QR with Wilkinson shift on one leaf (Algorithm
// 1's leaf solver; Golub & Van Loan Sec. 8.3), done in two phases so that the
// scalar bulge chase is not repeated by every lane of a warp (on this part a
// warp-wide FP64 instruction costs the FP64 pipe 16 cycles whatever it does):
//   k_leaf_qr     one thread per leaf: the QR iterations on (a, b), recording
//                 every Givens rotation (k, c, s) and the unsorted eigenvalues;
//   k_leaf_apply  one warp per leaf: Q = I, the rotations applied in order (lane
//                 = row of Q), then the eigenpairs sorted ascending and written.
// Both take the same operations in the same order as a single-warp solver; a
// leaf whose rotations exceed its buffer runs the single-warp solver
// (leaf_solve_warp) in phase two.
__device__ __forceinline__ void leaf_load(const LeafDesc& lf, const double* A, const double* Bc,
                                          double* a, double* b)
{
    const int n = lf.n, g0 = lf.g0;
    for (int i = 0; i < n; i++) a[i] = A[g0 + i];
    for (int i = 0; i < n - 1; i++) b[i] = Bc[g0 + i];
    if (!lf.first) a[0] -= fabs(Bc[g0 - 1]);
    if (!lf.last) a[n - 1] -= fabs(Bc[g0 + n - 1]);
}

// The QR iterations on (a, b); rot(k, c, s) is called for every rotation in
// order.  Returns false when the sweep cap is reached.
template <class Rot>
__device__ __forceinline__ bool leaf_qr(int n, double* a, double* b, Rot rot)
{
    int sweeps = 0;
    int h = n - 1;
    while (h > 0) {
        for (int i = 0; i < h; i++)
            if (fabs(b[i]) <= TD_EPS * (fabs(a[i]) + fabs(a[i + 1]))) b[i] = 0.0;
        while (h > 0 && b[h - 1] == 0.0) h--;
        if (h == 0) break;
        int l = h - 1;
        while (l > 0 && b[l - 1] != 0.0) l--;
        if (++sweeps > 30 * n) return false;
        double dd = 0.5 * (a[h - 1] - a[h]);
        double bh = b[h - 1];
        double sg = (dd >= 0.0) ? 1.0 : -1.0;
        double mu = a[h] - bh * bh / (dd + sg * hypot(dd, bh));
        double x = a[l] - mu, z = b[l];
        for (int k = l; k < h; k++) {
            // the rotation by one reciprocal square root (a few ulp, like hypot and
            // two divides, at a third of their FP64 instructions); hypot when the
            // squares would underflow
            double r, c = 1.0, s = 0.0;
            const double r2 = x * x + z * z;
            if (r2 > 1e-290) {
                const double inv = rsqrt(r2);
                r = r2 * inv;
                c = x * inv;
                s = -z * inv;
            } else {
                r = hypot(x, z);
                if (r != 0.0) { c = x / r; s = -z / r; }
            }
            if (k > l) b[k - 1] = r;
            double p = a[k], q = b[k], w = a[k + 1];
            a[k] = c * c * p - 2.0 * c * s * q + s * s * w;
            a[k + 1] = s * s * p + 2.0 * c * s * q + c * c * w;
            b[k] = c * s * (p - w) + (c * c - s * s) * q;
            if (k + 1 < h) {
                double e = b[k + 1];
                z = -s * e;
                b[k + 1] = c * e;
                x = b[k];
            }
            rot(k, c, s);
        }
    }
    return true;
}

// Selection sort of the eigenvalues (ascending) with the matching columns of
// Q, then the leaf's outputs.  a: eigenvalues (every lane holds a copy).
__device__ __forceinline__ void leaf_finish(const LeafDesc& lf, double* a, double (*Q)[33], int lane)
{
    const int n = lf.n;
    for (int i = 0; i < n - 1; i++) {
        int m = i;
        for (int j = i + 1; j < n; j++) if (a[j] < a[m]) m = j;
        if (m != i) {
            double t = a[i]; a[i] = a[m]; a[m] = t;
            double u = Q[lane][i]; Q[lane][i] = Q[lane][m]; Q[lane][m] = u;
        }
    }
    __syncwarp();
    if (lane < n) {
        for (int c = 0; c < n; c++) lf.qout[(int64_t)c * n + lane] = Q[lane][c];
        double v = 0.0;
        for (int i = 0; i < n; i++) if (i == lane) v = a[i];
        lf.lam_out[lane] = lf.scale_ptr ? v * (*lf.scale_ptr) : v;
    }
}

// One leaf by one warp: every lane runs the chase, lane = row of Q.
__device__ void leaf_solve_warp(const LeafDesc& lf, const double* A, const double* Bc,
                                double (*Q)[33], int lane, int* status)
{
    double a[32], b[32];
    leaf_load(lf, A, Bc, a, b);
    for (int c = 0; c < 32; c++) Q[lane][c] = (lane == c) ? 1.0 : 0.0;
    __syncwarp();
    const bool ok = leaf_qr(lf.n, a, b, [&](int k, double c, double s) {
        double qk = Q[lane][k], qk1 = Q[lane][k + 1];
        Q[lane][k] = c * qk - s * qk1;
        Q[lane][k + 1] = s * qk + c * qk1;
    });
    if (!ok && lane == 0) atomicOr(status, TD_STATUS_LEAF);
    leaf_finish(lf, a, Q, lane);
}

__global__ void __launch_bounds__(128) k_leaf_qr(const LeafDesc* L, int nleaves, const double* A,
                                                 const double* Bc, LeafRot R, int* status)
{
    const int leaf = blockIdx.x * blockDim.x + threadIdx.x;
    if (leaf >= nleaves) return;
    const LeafDesc lf = L[leaf];
    double a[32], b[32];
    leaf_load(lf, A, Bc, a, b);
    const int64_t off = lf.rot_off;
    const int cap = lf.rot_cap;
    int nr = 0;
    const bool ok = leaf_qr(lf.n, a, b, [&](int k, double c, double s) {
        if (nr < cap) {
            R.c[off + nr] = c;
            R.s[off + nr] = s;
            R.k[off + nr] = (unsigned char)k;
        }
        nr++;
    });
    if (!ok) atomicOr(status, TD_STATUS_LEAF);
    R.n[leaf] = nr;
    for (int i = 0; i < lf.n; i++) lf.lam_out[i] = a[i];   // unsorted, unscaled
}

__global__ void __launch_bounds__(32 * LEAF_WARPS) k_leaf_apply(const LeafDesc* L, int nleaves,
                                                                const double* A, const double* Bc,
                                                                LeafRot R, int* status)
{
    __shared__ double Qs[LEAF_WARPS][32][33];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int leaf = blockIdx.x * LEAF_WARPS + wib;
    if (leaf >= nleaves) return;
    const LeafDesc lf = L[leaf];
    double (*Q)[33] = Qs[wib];
    const int nr = R.n[leaf];
    if (nr > lf.rot_cap) {   // rotations did not fit: the single-warp solver
        leaf_solve_warp(lf, A, Bc, Q, lane, status);
        return;
    }
    for (int c = 0; c < 32; c++) Q[lane][c] = (lane == c) ? 1.0 : 0.0;
    __syncwarp();
    // Rotations in chunks of 32, one per lane (coalesced), the next chunk
    // loaded while the current one is broadcast by shuffles and applied.
    const int64_t off = lf.rot_off;
    double cn = 0.0, sn = 0.0;
    int kn = 0;
    if (lane < nr) { cn = R.c[off + lane]; sn = R.s[off + lane]; kn = R.k[off + lane]; }
    for (int r0 = 0; r0 < nr; r0 += 32) {
        const double cl = cn, sl = sn;
        const int kl = kn;
        const int m = min(32, nr - r0);
        if (r0 + 32 + lane < nr) {
            cn = R.c[off + r0 + 32 + lane]; sn = R.s[off + r0 + 32 + lane]; kn = R.k[off + r0 + 32 + lane];
        }
        for (int j = 0; j < m; j++) {
            const int k = __shfl_sync(0xffffffffu, kl, j);
            const double c = __shfl_sync(0xffffffffu, cl, j);
            const double s = __shfl_sync(0xffffffffu, sl, j);
            double qk = Q[lane][k], qk1 = Q[lane][k + 1];
            Q[lane][k] = c * qk - s * qk1;
            Q[lane][k + 1] = s * qk + c * qk1;
        }
    }
    double a[32];
    for (int i = 0; i < lf.n; i++) a[i] = lf.lam_out[i];
    __syncwarp();   // every lane has read the unsorted eigenvalues before they are overwritten
    leaf_finish(lf, a, Q, lane);
}

void td_launch_leaf(const LeafDesc* leaves, int nleaves, const double* A, const double* Bc,
                    const LeafRot& R, int* status, cudaStream_t st)
{
    if (nleaves <= 0) return;
    td_prof_begin(st); k_leaf_qr<<<td_cdiv(nleaves, 128), 128, 0, st>>>(leaves, nleaves, A, Bc, R, status); td_prof_end(st, "k_leaf_qr");
    td_prof_begin(st); k_leaf_apply<<<td_cdiv(nleaves, LEAF_WARPS), 32 * LEAF_WARPS, 0, st>>>(leaves, nleaves, A, Bc, R, status); td_prof_end(st, "k_leaf_apply");
}

// ---------------------------------------------------------------------------
// Block reductions / scans (blockDim.x = PREP_NT)
// ---------------------------------------------------------------------------
#define PREP_NT 512
__device__ double blk_sum(double v, double* red)
{
    v = td_warp_sum(v);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) r += red[i];
    return r;
}

__device__ double blk_max(double v, double* red)
{
    v = td_warp_max(v);
    int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double r = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) r = fmax(r, red[i]);
    return r;
}

// exclusive scan of a 0/1 flag over the block; returns prefix, *total = block total
__device__ int blk_scan(int f, int* red, int* total)
{
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned bal = __ballot_sync(0xffffffffu, f);
    int pre = __popc(bal & ((1u << lane) - 1u));
    __syncthreads();
    if (lane == 0) red[w] = __popc(bal);
    __syncthreads();
    int base = 0, tot = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) {
        if (i < w) base += red[i];
        tot += red[i];
    }
    *total = tot;
    return base + pre;
}

// s + c += a with s carrying the rounded sum and c the accumulated rounding
// errors (Knuth's TwoSum; Ogita, Rump & Oishi's compensated summation).
__device__ __forceinline__ void cs_add(double& s, double& c, double a)
{
    const double t = __dadd_rn(s, a);
    const double bp = __dsub_rn(t, s);
    const double err = __dadd_rn(__dsub_rn(s, __dsub_rn(t, bp)), __dsub_rn(a, bp));
    s = t;
    c = __dadd_rn(c, err);
}

// sum over the block of the thread values (s, c), rounded once at the end:
// the sum as if computed in twice the working precision, then rounded, which
// is the correctly rounded sum except within ~n^2 eps^2 of a rounding
// boundary (whatever the order of the terms).
__device__ double blk_sum_compensated(double s, double c, double* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double s2 = __shfl_xor_sync(0xffffffffu, s, o);
        const double c2 = __shfl_xor_sync(0xffffffffu, c, o);
        cs_add(s, c, s2);
        c = __dadd_rn(c, c2);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) { red[2 * w] = s; red[2 * w + 1] = c; }
    __syncthreads();
    double ts = red[0], tc = red[1];
    for (int i = 1; i < (int)(blockDim.x >> 5); i++) {
        cs_add(ts, tc, red[2 * i]);
        tc = __dadd_rn(tc, red[2 * i + 1]);
    }
    return __dadd_rn(ts, tc);
}

// ---------------------------------------------------------------------------
// k_prep: one CTA per merge.  eq. T3 (u from Q1's last row and Q2's first row,
// rho = |b_k|, sign folded into u), stable merge of D1 and D2, normalisation of
// u (rho absorbs |u|^2), deflation, compaction of the survivors.
// Deflation reading (Gu & Eisenstat): tau = 8 eps max(max|d|, rho max|z|);
// sweep ascending against the last survivor j: rho|z_i| <= tau deflates i;
// else with r = sqrt(z_i^2 + z_j^2), c = z_i/r, s = z_j/r, |(d_i - d_j) c s|
// <= tau rotates the pair (z_j -> 0, z_i -> r) and deflates j.
// The decisions are a function of the inputs alone: |z|^2 is summed with
// compensation (the correctly rounded sum but for ties within ~n^2 eps^2),
// and every operation of the sweep is rounded once as written (no fused
// multiply-add): for nearly equal poles t is a few ulp, so a differently
// rounded rotated pole would change later decisions.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PREP_NT) k_prep(const MergeDesc* M, LevelWS ws)
{
    __shared__ double red[32];
    __shared__ double red2[2 * (PREP_NT / 32)];
    __shared__ int ired[32];
    __shared__ double s_tau, s_rho;
    MergeDesc md = M[blockIdx.x];
    const int n = md.n, n1 = md.n1, n2 = n - n1, g0 = md.g0;
    const double* lam = md.lam_in;
    const double beta = *md.beta_ptr;
    const double sgn = (beta < 0.0) ? -1.0 : 1.0;
    double zz = 0.0, zzc = 0.0, dmax = 0.0, zmax = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double v = lam[i], z;
        int r;
        if (i < n1) {
            int lo = 0, hi = n2;   // count of D2 < v
            while (lo < hi) { int mid = (lo + hi) >> 1; if (lam[n1 + mid] < v) lo = mid + 1; else hi = mid; }
            r = i + lo;
            z = md.z1 ? md.z1[i] : md.qin1[(int64_t)i * n1 + (n1 - 1)];
        } else {
            int j = i - n1;
            int lo = 0, hi = n1;   // count of D1 <= v
            while (lo < hi) { int mid = (lo + hi) >> 1; if (lam[mid] <= v) lo = mid + 1; else hi = mid; }
            r = j + lo;
            z = sgn * (md.z2 ? md.z2[j] : md.qin2[(int64_t)j * n2]);
        }
        ws.dsort[g0 + r] = v;
        ws.zsort[g0 + r] = z;
        ws.src[g0 + r] = i;
        // z^2 = p + e exactly (e from a fused multiply-add), both summed
        const double p = __dmul_rn(z, z);
        cs_add(zz, zzc, p);
        zzc = __dadd_rn(zzc, fma(z, z, -p));
        dmax = fmax(dmax, fabs(v));
        zmax = fmax(zmax, fabs(z));
    }
    zz = blk_sum_compensated(zz, zzc, red2);
    dmax = blk_max(dmax, red);
    zmax = blk_max(zmax, red);
    double nrm = sqrt(zz);
    double rho = fabs(beta);
    if (nrm > 0.0) {
        rho *= nrm * nrm;
        zmax /= nrm;
    }
    __syncthreads();
    if (nrm > 0.0)
        for (int i = threadIdx.x; i < n; i += blockDim.x) ws.zsort[g0 + i] /= nrm;
    if (threadIdx.x == 0) {
        s_tau = 8.0 * TD_EPS * fmax(dmax, rho * zmax);
        s_rho = rho;
    }
    __syncthreads();

    // Deflation sweep by the whole CTA, PREP_NT entries per batch.  The sweep's
    // only carried state is the last survivor (index, d, z, support mask): entry
    // i either deflates by type 1 (independent of the state), or is tested
    // against the state and becomes the new survivor (after a rotation when the
    // test holds).  Each thread decides its entry against its predecessor's
    // current final state (exchanged through shared memory) and the batch
    // repeats until no decision changes: since every decision depends only on
    // the predecessor's, round k settles the first k candidates, so the fixpoint
    // (reached in at most PREP_NT + 1 rounds, typically 2) is exactly the
    // sequential sweep, with the same arithmetic per decision.  A warp alone
    // (32 entries per batch) used one of the SM's four FP64 units and spent most
    // of a batch in latency.
    // A thread recomputes only in the first round and after its predecessor's
    // state changed (the decision is a function of that state alone).  A pair is
    // sent to the exact test (the square root and divides, which cost most of a
    // round on the 1/64-rate FP64 pipe) only when a cheap bound cannot exclude
    // the rotation: with S = z_i^2 + z_j^2 the exact |t c s| is |t z_i z_j| / S,
    // every operation of the test is rounded once, so the computed |t c s| is at
    // least (1 - 9 eps) of it; the bound |t z_i z_j| > tau S (1 + 1e-12), itself
    // computed with a few roundings, therefore implies no rotation.  Decisions
    // are those of the exact test alone.  States are compared as bit patterns
    // (an FP64 compare issues on the FP64 pipe).
    {
        __shared__ double s_fd[2][PREP_NT], s_fz[2][PREP_NT];
        __shared__ int s_fm[2][PREP_NT];
        __shared__ int s_ch[2][PREP_NT];
        __shared__ int s_lastc[PREP_NT / 32], s_rotw[PREP_NT / 32];
        __shared__ int s_j, s_mj;
        __shared__ double s_dj, s_zj;
        const unsigned FULL = 0xffffffffu;
        const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
        const unsigned below = (1u << lane) - 1u;
        const double tau = s_tau;
        if (tid == 0) { s_j = -1; s_mj = 0; s_dj = 0.0; s_zj = 0.0; }
        int nrot = 0;
        __syncthreads();
        for (int base = 0; base < n; base += PREP_NT) {
            const int i = base + tid;
            const bool valid = i < n;
            const double d0 = valid ? ws.dsort[g0 + i] : 0.0;
            const double z0 = valid ? ws.zsort[g0 + i] : 0.0;
            const int m0 = valid ? ((ws.src[g0 + i] < n1) ? 1 : 2) : 0;
            const bool type1 = valid && (rho * fabs(z0) <= tau);
            const bool cand = valid && !type1;
            const unsigned cmask = __ballot_sync(FULL, cand);
            if (lane == 0) s_lastc[w] = cmask ? w * 32 + 31 - __clz(cmask) : -1;
            const int j = s_j, mj = s_mj;      // carried survivor
            const double dj = s_dj, zj = s_zj;
            double fd = d0, fz = z0, c = 0.0, sn = 0.0, djn = 0.0;
            int fm = m0;
            bool rot = false;
            s_fd[0][tid] = fd; s_fz[0][tid] = fz; s_fm[0][tid] = fm; s_ch[0][tid] = 1;
            __syncthreads();
            // predecessor: the last candidate before this entry in the batch (-1:
            // the carried survivor)
            const unsigned pm = cmask & below;
            int pl = pm ? w * 32 + 31 - __clz(pm) : -1;
            for (int v = w - 1; pl < 0 && v >= 0; v--) pl = s_lastc[v];
            const bool has_pred = pl >= 0 || j >= 0;
            int last = -1;   // the batch's last candidate
            for (int v = PREP_NT / 32 - 1; last < 0 && v >= 0; v--) last = s_lastc[v];
            for (int it = 0; it <= PREP_NT; it++) {
                const int b = it & 1;
                double pd = dj, pz = zj;
                int pmk = mj, pch = 0;
                if (pl >= 0) { pd = s_fd[b][pl]; pz = s_fz[b][pl]; pmk = s_fm[b][pl]; pch = s_ch[b][pl]; }
                bool nr = rot;
                double nd = fd, nz = fz, nc = c, ns = sn, nj = djn;
                int nm = fm;
                if (it == 0 || pch) {
                    nr = false;
                    nd = d0; nz = z0; nc = 0.0; ns = 0.0; nj = 0.0;
                    nm = m0;
                    if (cand && has_pred) {
                        const double t = d0 - pd;
                        const bool maybe = !(fabs(t) * fabs(z0) * fabs(pz) >
                                             tau * (z0 * z0 + pz * pz) * (1.0 + 1e-12));
                        if (maybe) {
                            // survivors' weights: rho |z| > tau >= 8 eps rho max|z|, so
                            // the squares neither underflow nor overflow
                            const double r = sqrt(__dadd_rn(__dmul_rn(z0, z0), __dmul_rn(pz, pz)));
                            const double cc = z0 / r, ss = pz / r;
                            if (fabs(__dmul_rn(__dmul_rn(t, cc), ss)) <= tau) {
                                nr = true;
                                const double c2 = __dmul_rn(cc, cc), s2 = __dmul_rn(ss, ss);
                                nj = __dadd_rn(__dmul_rn(c2, pd), __dmul_rn(s2, d0));
                                nd = __dadd_rn(__dmul_rn(s2, pd), __dmul_rn(c2, d0));
                                nz = r;
                                nm = m0 | pmk;
                                nc = cc;
                                ns = ss;
                            }
                        }
                    }
                }
                const bool changed = nr != rot || nm != fm ||
                                     __double_as_longlong(nd) != __double_as_longlong(fd) ||
                                     __double_as_longlong(nz) != __double_as_longlong(fz);
                rot = nr; fd = nd; fz = nz; fm = nm; c = nc; sn = ns; djn = nj;
                s_fd[b ^ 1][tid] = fd; s_fz[b ^ 1][tid] = fz; s_fm[b ^ 1][tid] = fm;
                s_ch[b ^ 1][tid] = changed;
                if (!__syncthreads_or(changed)) break;
            }
            if (type1) { ws.zsort[g0 + i] = 0.0; ws.keep[g0 + i] = 0; }
            if (cand) { ws.keep[g0 + i] = fm; ws.dsort[g0 + i] = fd; ws.zsort[g0 + i] = fz; }
            const unsigned rmask = __ballot_sync(FULL, rot);
            if (lane == 0) s_rotw[w] = __popc(rmask);
            // the predecessor's own entry is written above (by another warp,
            // possibly): its deflation below must come after
            __syncthreads();
            int rbefore = 0, rtotal = 0;
            for (int v = 0; v < PREP_NT / 32; v++) {
                rbefore += (v < w) ? s_rotw[v] : 0;
                rtotal += s_rotw[v];
            }
            if (rot) {
                // the predecessor deflates: rotated d, zero z; rotations keep sweep order
                const int pj = pl >= 0 ? base + pl : j;
                const int slot = nrot + rbefore + __popc(rmask & below);
                ws.dsort[g0 + pj] = djn;
                ws.zsort[g0 + pj] = 0.0;
                ws.keep[g0 + pj] = 0;
                ws.rot_j[g0 + slot] = pj;
                ws.rot_i[g0 + slot] = i;
                ws.rot_c[g0 + slot] = c;
                ws.rot_s[g0 + slot] = sn;
            }
            nrot += rtotal;
            if (tid == last) { s_j = i; s_dj = fd; s_zj = fz; s_mj = fm; }
            __syncthreads();
        }
        if (tid == 0) ws.nrot[blockIdx.x] = nrot;
    }
    __syncthreads();

    // compaction of survivors and deflated indices
    int run_k = 0, run_d = 0;
    for (int base = 0; base < n; base += blockDim.x) {
        int i = base + threadIdx.x;
        int f = (i < n) ? ws.keep[g0 + i] : 0;
        int tot;
        int pre = blk_scan(f, ired, &tot);
        int nvalid = min((int)blockDim.x, n - base);
        if (i < n) {
            if (f) {
                int k = run_k + pre;
                double zi = ws.zsort[g0 + i];
                ws.survIdx[g0 + k] = i;
                const double di = ws.dsort[g0 + i], wi = s_rho * zi * zi;
                ws.dK[g0 + k] = di;
                ws.zK[g0 + k] = zi;
                ws.wK[g0 + k] = wi;
                const float dh = __double2float_rn(di);
                ws.dhK[g0 + k] = dh;
                const double r1 = di - (double)dh;   // exact
                const float dm = __double2float_rn(r1);
                ws.dlK[g0 + k] = dm;
                ws.dxK[g0 + k] = __double2float_rn(r1 - (double)dm);   // exact (a few bits)
                const float wh = __double2float_rn(wi);
                ws.wfK[g0 + k] = wh;
                ws.wlK[g0 + k] = __double2float_rn(wi - (double)wh);
            } else {
                int l = run_d + ((int)threadIdx.x - pre);
                ws.deflIdx[g0 + l] = i;
            }
        }
        run_k += tot;
        run_d += nvalid - tot;
        __syncthreads();
    }
    // order of the survivors in the update product: support 1, then 3, then 2
    const int K = run_k;
    int c1 = 0, c3 = 0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        int t = ws.keep[g0 + ws.survIdx[g0 + k]];
        c1 += (t == 1);
        c3 += (t == 3);
    }
    const int K1 = (int)blk_sum((double)c1, red);
    const int Km = (int)blk_sum((double)c3, red);
    int run1 = 0, run3 = 0, run2 = 0;
    for (int base = 0; base < K; base += blockDim.x) {
        int k = base + threadIdx.x;
        int t = (k < K) ? ws.keep[g0 + ws.survIdx[g0 + k]] : 0;
        int tot1, tot3, tot2;
        int p1 = blk_scan(t == 1, ired, &tot1);
        int p3 = blk_scan(t == 3, ired, &tot3);
        int p2 = blk_scan(t == 2, ired, &tot2);
        if (k < K) {
            int p = (t == 1) ? run1 + p1 : (t == 3) ? K1 + run3 + p3 : K1 + Km + run2 + p2;
            ws.gemmCol[g0 + p] = k;
            ws.gemmW[g0 + p] = ws.survIdx[g0 + k];
        }
        run1 += tot1;
        run3 += tot3;
        run2 += tot2;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ws.K[blockIdx.x] = K;
        ws.rho[blockIdx.x] = s_rho;
        ws.kgrp[2 * blockIdx.x] = K1;
        ws.kgrp[2 * blockIdx.x + 1] = Km;
    }
}

// W[:, c] = column src[c] of diag(Q1, Q2) for the sorted order c, with the
// deflation rotations applied: one pass that reads each source column once and
// writes each W column once.
// Structure used: the sweep visits i in ascending order and rotates it against
// the last survivor j < i, so the rotations come sorted by i, and a chain
// (a maximal run whose j is the previous rotation's i) covers an interval of
// columns that no other chain enters (the columns strictly inside a chain that
// are not its i's are type-1 deflations, which no rotation touches).  A row
// visits its columns in ascending order holding the latest value of the
// chain's current j in a register: at a chain's first j the source value is
// held; at each i the pair is rotated, the j column stored and the rotated i
// held (stored when the chain ends); every other column is a plain copy.
// Grid: (merge, 256-row tile, BW_G column groups); group boundaries are moved
// forward out of chains, so each group applies whole chains.  The control flow
// depends only on the column and the rotation list: it is uniform in a CTA.
#define BW_NT 256
#define BW_G 32
#define BW_U 8   // source columns loaded ahead of their use

// The smallest b' >= b that no chain straddles (no chain has its first j below
// b' and a later column at or above it).
__device__ int bw_boundary(const LevelWS& ws, int g0, int nrot, int n, int b)
{
    if (b >= n) return n;
    int lo = 0, hi = nrot;   // first rotation with i >= b
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (ws.rot_i[g0 + mid] < b) lo = mid + 1; else hi = mid;
    }
    if (lo >= nrot) return b;
    int st = lo;             // start of its chain
    while (st > 0 && ws.rot_j[g0 + st] == ws.rot_i[g0 + st - 1]) st--;
    if (ws.rot_j[g0 + st] >= b) return b;
    int e = lo;              // end of the chain
    while (e + 1 < nrot && ws.rot_j[g0 + e + 1] == ws.rot_i[g0 + e]) e++;
    return min(n, ws.rot_i[g0 + e] + 1);
}

__global__ void __launch_bounds__(BW_NT) k_build_w(const MergeDesc* M, LevelWS ws)
{
    const MergeDesc md = M[blockIdx.x];
    const int n = md.n, n1 = md.n1, n2 = n - n1, g0 = md.g0;
    const int G = min(BW_G, (n + 63) / 64);
    const int r = (int)blockIdx.y * BW_NT + (int)threadIdx.x;
    if ((int)blockIdx.z >= G || (int)blockIdx.y * BW_NT >= n) return;
    const bool live = r < n;
    const int nrot = ws.nrot[blockIdx.x];
    __shared__ int s_cb, s_ce, s_t;
    if (threadIdx.x == 0) {
        const int cb = bw_boundary(ws, g0, nrot, n, (int)(((int64_t)blockIdx.z * n) / G));
        const int ce = bw_boundary(ws, g0, nrot, n, (int)(((int64_t)(blockIdx.z + 1) * n) / G));
        int lo = 0, hi = nrot;   // first rotation with i >= cb
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (ws.rot_i[g0 + mid] < cb) lo = mid + 1; else hi = mid;
        }
        s_cb = cb; s_ce = ce; s_t = lo;
    }
    __syncthreads();
    const int cb = s_cb, ce = s_ce;
    int t = s_t;
    int rj = n, ri = n;
    double rc = 1.0, rs = 0.0;
    if (t < nrot) { rj = ws.rot_j[g0 + t]; ri = ws.rot_i[g0 + t]; rc = ws.rot_c[g0 + t]; rs = ws.rot_s[g0 + t]; }
    double* const W = md.W;
    int cj = -1;      // column whose latest value is held in cv
    double cv = 0.0;
    for (int c0 = cb; c0 < ce; c0 += BW_U) {
        double q[BW_U];
#pragma unroll
        for (int u = 0; u < BW_U; u++) {
            const int c = c0 + u;
            double v = 0.0;
            if (live && c < ce) {
                // src is a permutation of [0, n) for ordered input; the clamp keeps a
                // non-finite input (reported as TDEIG_EINVAL) from indexing outside.
                const int sc = min(max(ws.src[g0 + c], 0), n - 1);
                if (sc < n1) { if (r < n1) v = md.qin1[(int64_t)sc * n1 + r]; }
                else if (r >= n1) v = md.qin2[(int64_t)(sc - n1) * n2 + (r - n1)];
            }
            q[u] = v;
        }
#pragma unroll
        for (int u = 0; u < BW_U; u++) {
            const int c = c0 + u;
            if (c >= ce) break;
            if (c == ri) {
                // rotation (j, i): the held j against this source column
                const double qj = cv, qi = q[u];
                // cj >= 0: the group holds its chains' first columns (a malformed
                // rotation list still writes nothing outside W)
                if (live && cj >= 0) W[(int64_t)cj * n + r] = rc * qj - rs * qi;
                cv = rs * qj + rc * qi;
                cj = c;
                t++;
                rj = n; ri = n;
                if (t < nrot) { rj = ws.rot_j[g0 + t]; ri = ws.rot_i[g0 + t]; rc = ws.rot_c[g0 + t]; rs = ws.rot_s[g0 + t]; }
                if (rj != c) {   // the chain ends here
                    if (live) W[(int64_t)c * n + r] = cv;
                    cj = -1;
                }
            } else if (c == rj) {
                cv = q[u];       // first j of a chain
                cj = c;
            } else if (live) {
                W[(int64_t)c * n + r] = q[u];
            }
        }
    }
}

int td_binary_version(int* out)
{
    cudaFuncAttributes a;
    if (cudaFuncGetAttributes(&a, k_prep) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    *out = a.binaryVersion;
    return 0;
}

void td_launch_prep(const MergeDesc* M, int nmerge, const LevelWS& ws, cudaStream_t st)
{
    td_prof_begin(st); k_prep<<<nmerge, PREP_NT, 0, st>>>(M, ws); td_prof_end(st, "k_prep");
}

void td_launch_merge_level(const MergeDesc* M, int nmerge, int nmax, int rows, int total_tiles,
                           const LevelWS& ws, int* status, int use_hss_mask, cudaStream_t st)
{
    (void)rows; (void)total_tiles; (void)status; (void)use_hss_mask;
    td_prof_begin(st); k_prep<<<nmerge, PREP_NT, 0, st>>>(M, ws); td_prof_end(st, "k_prep");
    dim3 gw(nmerge, td_cdiv(nmax, BW_NT), BW_G);
    td_prof_begin(st); k_build_w<<<gw, BW_NT, 0, st>>>(M, ws); td_prof_end(st, "k_build_w");
}

// ---------------------------------------------------------------------------
// Secular equation, one warp per root (Theorem 1).  Same iteration as the
// oracle: origin at the nearer pole (sign of f at the midpoint), unknown
// tau = lambda - d_origin, two-pole rational model of psi (poles <= i) and phi
// (poles > i) fitted in value and slope (Bunch, Nielsen & Sorensen), bisection
// when the model step leaves the bracket; it starts from the root of a
// two-pole model built from the midpoint value (the oracle starts at the
// middle of the bracket) and takes a model step below 1e-9 of tau as the
// converged value without evaluating there (the oracle evaluates once more).
// The K-term sums are lane-strided and reduced with warp shuffles.
// ---------------------------------------------------------------------------

// x = m 2^e with m in [1, 2) (sign kept): returns m and adds sgn * e to *ex.
// Zero (and subnormal) x is returned unchanged.
__device__ __forceinline__ double td_renorm(double x, int* ex, int sgn)
{
    const long long b = __double_as_longlong(x);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) return x;
    *ex += sgn * (e - 1023);
    return __longlong_as_double((b & ~(0x7ffLL << 52)) | (1023LL << 52));
}

__device__ __forceinline__ float td_rcp_f32(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ---- double-float (FP32 pair, value = hi + lo, about 48 bits) helpers -----
// a + b = s + e exactly (Knuth's TwoSum; no products, so nothing is contracted).
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// One term w_j / (delta_j - tau) of a secular sum in double-float, added to
// (sh, sl), its derivative term w_j / (delta_j - tau)^2 to sd in FP32 (the
// derivatives only scale the model step).  delta_j = d_j - d_org comes from the
// FP32 pairs of d (dh_j - dh_org is exact, the rest carries the 48-bit
// representation error of d, about 2^-48 |d| absolute), except for the near
// pole, whose exact FP64 difference from tau the caller passes as (xh, xl):
// every other pole is at least one pole gap from tau, so each term keeps a
// relative error of about 2^-46 when the poles are not clustered.
__device__ __forceinline__ void df_term(float dhj, float dlj, float oh, float ol, float th,
                                        float tl, float wh, float wl, bool nearp, float xh,
                                        float xl, float& sh, float& sl, float& sd)
{
    float Dh, Dl;
    if (nearp) {
        Dh = xh;
        Dl = xl;
    } else {
        float s1, e1, s2, e2;
        df_two_sum(dhj, -oh, s1, e1);
        df_two_sum(s1, -th, s2, e2);
        const float lo = __fadd_rn(__fadd_rn(e1, __fsub_rn(dlj, ol)), __fsub_rn(e2, tl));
        Dh = __fadd_rn(s2, lo);
        Dl = __fsub_rn(lo, __fsub_rn(Dh, s2));
    }
    // 1 / D = q (1 + r + ...), r = 1 - D q from the approximate reciprocal q
    const float q = td_rcp_f32(Dh);
    float r = fmaf(-Dh, q, 1.0f);
    r = fmaf(-Dl, q, r);
    const float ql = q * r;
    const float Th = wh * q;
    const float Tl = fmaf(wh, q, -Th) + fmaf(wh, ql, wl * q);
    float t, e;
    df_two_sum(sh, Th, t, e);
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(e, Tl));
    sd = fmaf(Th, q, sd);
}

__device__ __forceinline__ void df_warp_sum(float& h, float& l)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o);
        const float ol = __shfl_xor_sync(0xffffffffu, l, o);
        float t, e;
        df_two_sum(h, oh, t, e);
        h = t;
        l = __fadd_rn(l, __fadd_rn(e, ol));
    }
}

// The model step of the iteration (Bunch, Nielsen & Sorensen's two-pole
// rational model of psi (poles <= i) and phi (poles > i) fitted in value and
// slope at tau; for the last root one pole): returns tau + step when the model
// root lies inside the bracket (lo, hi), else the bracket's midpoint.  Its
// divide is a reciprocal by td_recip (a few ulp): the step only proposes the
// next point, and a step accepted without another evaluation is below 1e-9 of
// tau, so its last-place error is far below tau's.
__device__ __forceinline__ double secular_step(double f, double dpsi, double dphi, double tau,
                                               double lo, double hi, double deli, double deli1,
                                               bool last, double* step_out, bool* model_out)
{
    const double a1 = deli - tau;
    double step = 0.0;
    bool ok = true;
    if (!last) {
        const double a2 = deli1 - tau;
        const double E = f - dpsi * a1 - dphi * a2;
        const double beta = E * (a1 + a2) + dpsi * a1 * a1 + dphi * a2 * a2;
        const double c0 = a1 * a2 * f;
        double disc = beta * beta - 4.0 * E * c0;
        if (disc < 0.0) disc = 0.0;
        const double den = beta + (beta >= 0.0 ? sqrt(disc) : -sqrt(disc));
        if (den == 0.0) ok = false; else step = 2.0 * c0 * td_recip(den);
    } else {
        const double E = f - dpsi * a1;
        if (E == 0.0) ok = false; else step = a1 * f * td_recip(E);
    }
    const bool model = ok && tau + step > lo && tau + step < hi;
    *step_out = step;
    *model_out = model;
    return model ? tau + step : 0.5 * (lo + hi);
}

// Merges with K >= this many poles run the double-float iterations before the
// FP64 ones: below it the lane-0 scalar work of an iteration (FP64 issue costs a
// whole warp slot whatever the active lanes, ~40 slots for the model step) is
// not small next to an FP64 sum (14 slots per 32 terms).
#define TD_SECULAR_DF_MINK 256
#define TD_SECULAR_DF_MAXIT 16

// One root of the secular equation by one warp (Theorem 1; Remark 1 for gamma
// and mu).  dh, dl, wf, wl: d and w as FP32 pairs.
//   Origin: the midpoint value that picks the origin pole and seeds the start
//   is taken in FP32 (about 1/50 of the cost of an FP64 evaluation here) and
//   the bracket is the whole interval on the origin's side, (0, d_i+1 - d_i) or
//   (-(d_i+1 - d_i), 0): a wrong sign from FP32 rounding can then only choose
//   the farther pole as origin for a root near the midpoint, where either
//   origin is accurate.
//   Start: the root of the two-pole model with the other terms frozen at their
//   midpoint value.
//   Double-float iterations (K >= TD_SECULAR_DF_MINK): the same safeguarded
//   model iteration on psi, phi summed in double-float (an FP32 pair per term,
//   ~30 FP32 operations, against ~14 FP64 issue slots per term on a part whose
//   FP64 rate is 1/64 of FP32), until f is within the double-float noise
//   (2^-40 of its scale) or the step is below 1e-12 of tau: tau is then within
//   ~1e-11 of the root.
//   FP64 iterations: the same iteration and stopping test as the oracle,
//   |f| <= 8 eps (1 + |psi| + |phi| + |tau| f'); a model step below 1e-9 of
//   tau is taken as converged without evaluating at the new point (the step is
//   second order in an error of that size).  After the double-float phase one
//   FP64 evaluation normally ends the root.
// *iters: FP64 evaluations; *df_iters: double-float evaluations.
__device__ void secular_root_warp(const double* __restrict__ d, const double* __restrict__ w, int K,
                                  int i, int lane, double* lam, double* gam, double* mu, int* iters,
                                  int* df_iters, const float* __restrict__ dh,
                                  const float* __restrict__ dl, const float* __restrict__ wf,
                                  const float* __restrict__ wl)
{
    *df_iters = 0;
    if (K == 1) { *lam = d[0] + w[0]; *gam = w[0]; *mu = 0.0; *iters = 0; return; }
    const bool last = (i == K - 1);
    int org;
    double lo, hi, fmid = 0.0;
    if (!last) {
        const double gap = d[i + 1] - d[i];
        const float hf = __double2float_rn(0.5 * gap);
        const float ohi = dh[i], olo = dl[i];
        float f = 0.0f;
        for (int j = lane; j < K; j += 32) {
            const float del = (dh[j] - ohi) + (dl[j] - olo);   // d_j - d_i
            f = fmaf(wf[j], td_rcp_f32(del - hf), f);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(0xffffffffu, f, o);
        fmid = 1.0 + (double)f;
        if (fmid >= 0.0) { org = i; lo = 0.0; hi = gap; }
        else { org = i + 1; lo = -gap; hi = 0.0; }
    } else {
        double zz = 0.0;
        for (int j = lane; j < K; j += 32) zz += w[j];
        zz = td_warp_sum(zz);
        org = i; lo = 0.0; hi = zz;
    }
    const double dorg = d[org];
    const double deli = d[i] - dorg;
    const double deli1 = last ? 0.0 : d[i + 1] - dorg;
    // The scalar work of the iteration (start, stopping tests, model step) is
    // done by lane 0 alone and the new tau and the decision broadcast: repeated
    // by 32 lanes it cost as much FP64 issue as the sums of a small merge.
    double tau = 0.5 * (lo + hi);
    if (!last && lane == 0) {
        // Start: 1 + c + w_i/(deli - t) + w_i1/(deli1 - t) = 0 with c the other
        // terms' midpoint value, a quadratic a t^2 - b t + c0 = 0 solved for its
        // root in the bracket (the midpoint is the fallback).
        const double mid = 0.5 * (d[i + 1] - d[i]);   // midpoint offset from d_i
        const double wi = w[i], wi1 = w[i + 1];
        const double rm = td_recip(mid);
        const double a = fmid + wi * rm - wi1 * rm;   // 1 + c
        const double b = a * (deli + deli1) + wi + wi1;
        const double c0 = a * deli * deli1 + wi * deli1 + wi1 * deli;
        const double disc = b * b - 4.0 * a * c0;
        if (disc >= 0.0) {
            const double qq = 0.5 * (b + (b >= 0.0 ? sqrt(disc) : -sqrt(disc)));
            double t0 = 0.5 * (lo + hi);
            bool got = false;
            if (qq != 0.0) {
                const double r1 = c0 * td_recip(qq);
                if (r1 > lo && r1 < hi) { t0 = r1; got = true; }
            }
            if (!got && a != 0.0) {
                const double r2 = qq * td_recip(a);
                if (r2 > lo && r2 < hi) t0 = r2;
            }
            tau = t0;
        }
    }
    tau = __shfl_sync(0xffffffffu, tau, 0);

    // ---- double-float iterations ------------------------------------------
    // Their bracket updates trust the sign of a double-float f, which clustered
    // poles (terms of poles other than the two nearest, at distances near the
    // 2^-48 |d| representation error) can get wrong; the FP64 iterations start
    // again from the whole bracket, so only the start can suffer from that.
    const double lo0 = lo, hi0 = hi;
    if (K >= TD_SECULAR_DF_MINK) {
        const float oh = dh[org], ol = dl[org];
        // the near pole other than the origin, and its exact offset from it
        const int jn = last ? -1 : (org == i ? i + 1 : i);
        const double djn = last ? 0.0 : d[jn] - dorg;
        int itdf = 0;
        for (; itdf < TD_SECULAR_DF_MAXIT; itdf++) {
            const float th = __double2float_rn(tau);
            const float tl = __double2float_rn(tau - (double)th);
            const double x = djn - tau;
            const float xh = __double2float_rn(x);
            const float xl = __double2float_rn(x - (double)xh);
            float ph = 0.0f, pl = 0.0f, pd = 0.0f, fh = 0.0f, fl = 0.0f, fd = 0.0f;
            for (int j = lane; j <= i; j += 32)
                df_term(dh[j], dl[j], oh, ol, th, tl, wf[j], wl[j], j == jn, xh, xl, ph, pl, pd);
            for (int j = i + 1 + lane; j < K; j += 32)
                df_term(dh[j], dl[j], oh, ol, th, tl, wf[j], wl[j], j == jn, xh, xl, fh, fl, fd);
            df_warp_sum(ph, pl);
            df_warp_sum(fh, fl);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                pd += __shfl_xor_sync(0xffffffffu, pd, o);
                fd += __shfl_xor_sync(0xffffffffu, fd, o);
            }
            int stop = 0;
            double nt = tau;
            if (lane == 0) {
                const double psi = (double)ph + (double)pl, phi = (double)fh + (double)fl;
                const double dpsi = pd, dphi = fd;
                const double f = 1.0 + psi + phi;
                const double noise = 9.094947017729282e-13 *   // 2^-40
                                     (1.0 + fabs(psi) + fabs(phi) + fabs(tau) * (dpsi + dphi));
                if (fabs(f) <= noise) {
                    stop = 1;
                } else {
                    if (f > 0.0) hi = tau; else lo = tau;
                    double step;
                    bool model;
                    nt = secular_step(f, dpsi, dphi, tau, lo, hi, deli, deli1, last, &step, &model);
                    if (hi - lo <= 4.0 * TD_EPS * fmax(fabs(lo), fabs(hi)) ||
                        (model && fabs(step) <= 1e-12 * fabs(tau)))
                        stop = 1;
                }
            }
            stop = __shfl_sync(0xffffffffu, stop, 0);
            tau = __shfl_sync(0xffffffffu, nt, 0);
            if (stop) { itdf++; break; }
        }
        *df_iters = itdf;
    }
    lo = lo0;
    hi = hi0;

    // ---- FP64 iterations ---------------------------------------------------
    int it;
    for (it = 1; it <= TD_SECULAR_MAXIT; it++) {
        double s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0;
        for (int j = lane; j <= i; j += 32) {
            double q = td_recip((d[j] - dorg) - tau);
            double t = w[j] * q;
            s1 += t; s2 += t * q;
        }
        for (int j = i + 1 + lane; j < K; j += 32) {
            double q = td_recip((d[j] - dorg) - tau);
            double t = w[j] * q;
            s3 += t; s4 += t * q;
        }
        const double psi = td_warp_sum(s1), dpsi = td_warp_sum(s2);
        const double phi = td_warp_sum(s3), dphi = td_warp_sum(s4);
        int stop = 0;
        double nt = tau;
        if (lane == 0) {
            const double f = 1.0 + psi + phi;
            const double err = 8.0 * TD_EPS * (1.0 + fabs(psi) + fabs(phi) + fabs(tau) * (dpsi + dphi));
            if (fabs(f) <= err) {
                stop = 1;
            } else {
                if (f > 0.0) hi = tau; else lo = tau;
                if (hi - lo <= 4.0 * TD_EPS * fmax(fabs(lo), fabs(hi))) {
                    stop = 1;
                } else {
                    double step;
                    bool model;
                    nt = secular_step(f, dpsi, dphi, tau, lo, hi, deli, deli1, last, &step, &model);
                    if (nt == tau) stop = 1;
                    // a model step below 1e-9 of tau: tau is within about that of the
                    // root and the step (second order in that error) lands within
                    // rounding of it, so nt is taken without another evaluation
                    else if (model && fabs(step) <= 1e-9 * fabs(tau)) stop = 2;
                }
            }
        }
        stop = __shfl_sync(0xffffffffu, stop, 0);
        if (stop == 1) break;
        tau = __shfl_sync(0xffffffffu, nt, 0);
        if (stop == 2) break;
    }
    *lam = dorg + tau;
    if (last) { *gam = tau; *mu = 0.0; }
    else if (org == i) { *gam = tau; *mu = (d[i + 1] - d[i]) - tau; }
    else { *mu = -tau; *gam = (d[i + 1] - d[i]) + tau; }
    *iters = it;
}

// ---------------------------------------------------------------------------
// Small merges (K <= 256): several roots per warp, one aligned group of G
// lanes per root (G = 4, 8 or 16).  The iteration, stopping tests and arithmetic
// per term are those of secular_root_warp; the sums run over the group and are
// reduced within it.  What a warp of one root spent on its scalar work (the
// model step and tests on lane 0, ~40 FP64 issue slots per iteration, each
// costing a whole warp slot on this part whatever the active lanes) and on
// five levels of FP64 shuffle sums is then shared by 32 / G roots: on the
// lowest levels of a batch (K of 30 to 200) that work, not the K-term sums,
// set the time.  Groups of one warp may belong to different merges and need
// different iteration counts, so every loop that holds a shuffle runs until
// no group of the warp needs it (finished groups idle through it).
// ---------------------------------------------------------------------------
template <int G>
__device__ __forceinline__ float grp_sum_f(float v)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <int G>
__device__ __forceinline__ double grp_sum_d(double v)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
template <int G>
__device__ __forceinline__ void grp_df_sum(float& h, float& l)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o);
        const float ol = __shfl_xor_sync(0xffffffffu, l, o);
        float t, e;
        df_two_sum(h, oh, t, e);
        h = t;
        l = __fadd_rn(l, __fadd_rn(e, ol));
    }
}

// One root per group of G lanes (gl: lane within the group).  act: the group
// has a root (i < K); all lanes of the warp must call together.
template <int G>
__device__ void secular_root_group(const double* __restrict__ d, const double* __restrict__ w,
                                   int K, int i, bool act, int gl, double* lam, double* gam,
                                   double* mu, int* iters, int* df_iters,
                                   const float* __restrict__ dh, const float* __restrict__ dl,
                                   const float* __restrict__ wf, const float* __restrict__ wl)
{
    const unsigned FULL = 0xffffffffu;
    *df_iters = 0;
    *iters = 0;
    const bool run = act && K > 1;   // K == 1: closed form, no sums
    const bool last = run && i == K - 1;
    int org = i;
    double lo = 0.0, hi = 0.0, fmid = 0.0;
    {
        // origin from the FP32 midpoint value (not the last root)
        const bool mid = run && !last;
        double gap = 0.0;
        float hf = 0.0f, ohi = 0.0f, olo = 0.0f;
        if (mid) {
            gap = d[i + 1] - d[i];
            hf = __double2float_rn(0.5 * gap);
            ohi = dh[i];
            olo = dl[i];
        }
        float f = 0.0f;
        const int ke = mid ? K : 0;
        for (int j = gl; j < ke; j += G) {
            const float del = (dh[j] - ohi) + (dl[j] - olo);   // d_j - d_i
            f = fmaf(wf[j], td_rcp_f32(del - hf), f);
        }
        f = grp_sum_f<G>(f);
        if (mid) {
            fmid = 1.0 + (double)f;
            if (fmid >= 0.0) { org = i; lo = 0.0; hi = gap; }
            else { org = i + 1; lo = -gap; hi = 0.0; }
        }
    }
    if (__any_sync(FULL, last)) {
        double zz = 0.0;
        const int ke = last ? K : 0;
        for (int j = gl; j < ke; j += G) zz += w[j];
        zz = grp_sum_d<G>(zz);
        if (last) { org = i; lo = 0.0; hi = zz; }
    }
    const double dorg = run ? d[org] : 0.0;
    const double deli = run ? d[i] - dorg : 0.0;
    const double deli1 = (run && !last) ? d[i + 1] - dorg : 0.0;
    double tau = 0.5 * (lo + hi);
    if (run && !last && gl == 0) {
        // start: the root in the bracket of the two-pole model with the other
        // terms frozen at their midpoint value (as secular_root_warp)
        const double mid = 0.5 * (d[i + 1] - d[i]);
        const double wi = w[i], wi1 = w[i + 1];
        const double rm = td_recip(mid);
        const double a = fmid + wi * rm - wi1 * rm;   // 1 + c
        const double b = a * (deli + deli1) + wi + wi1;
        const double c0 = a * deli * deli1 + wi * deli1 + wi1 * deli;
        const double disc = b * b - 4.0 * a * c0;
        if (disc >= 0.0) {
            const double qq = 0.5 * (b + (b >= 0.0 ? sqrt(disc) : -sqrt(disc)));
            double t0 = 0.5 * (lo + hi);
            bool got = false;
            if (qq != 0.0) {
                const double r1 = c0 * td_recip(qq);
                if (r1 > lo && r1 < hi) { t0 = r1; got = true; }
            }
            if (!got && a != 0.0) {
                const double r2 = qq * td_recip(a);
                if (r2 > lo && r2 < hi) t0 = r2;
            }
            tau = t0;
        }
    }
    tau = __shfl_sync(FULL, tau, 0, G);

    // ---- double-float iterations (as secular_root_warp) ------------------
    const double lo0 = lo, hi0 = hi;
    bool dfrun = run && K >= TD_SECULAR_DF_MINK;
    if (__any_sync(FULL, dfrun)) {
        float oh = 0.0f, ol = 0.0f;
        int jn = -1;
        double djn = 0.0;
        if (dfrun) {
            oh = dh[org];
            ol = dl[org];
            jn = last ? -1 : (org == i ? i + 1 : i);
            djn = last ? 0.0 : d[jn] - dorg;
        }
        int itdf = 0;
        for (int t = 0; t < TD_SECULAR_DF_MAXIT; t++) {
            if (!__any_sync(FULL, dfrun)) break;
            float th = 0.0f, tl = 0.0f, xh = 0.0f, xl = 0.0f;
            if (dfrun) {
                th = __double2float_rn(tau);
                tl = __double2float_rn(tau - (double)th);
                const double x = djn - tau;
                xh = __double2float_rn(x);
                xl = __double2float_rn(x - (double)xh);
            }
            float ph = 0.0f, pl = 0.0f, pd = 0.0f, fh = 0.0f, fl = 0.0f, fd = 0.0f;
            const int ie = dfrun ? i : -1, ke = dfrun ? K : 0;
            for (int j = gl; j <= ie; j += G)
                df_term(dh[j], dl[j], oh, ol, th, tl, wf[j], wl[j], j == jn, xh, xl, ph, pl, pd);
            for (int j = i + 1 + gl; j < ke; j += G)
                df_term(dh[j], dl[j], oh, ol, th, tl, wf[j], wl[j], j == jn, xh, xl, fh, fl, fd);
            grp_df_sum<G>(ph, pl);
            grp_df_sum<G>(fh, fl);
            pd = grp_sum_f<G>(pd);
            fd = grp_sum_f<G>(fd);
            int stop = 0;
            double nt = tau;
            if (dfrun && gl == 0) {
                const double psi = (double)ph + (double)pl, phi = (double)fh + (double)fl;
                const double dpsi = pd, dphi = fd;
                const double f = 1.0 + psi + phi;
                const double noise = 9.094947017729282e-13 *   // 2^-40
                                     (1.0 + fabs(psi) + fabs(phi) + fabs(tau) * (dpsi + dphi));
                if (fabs(f) <= noise) {
                    stop = 1;
                } else {
                    if (f > 0.0) hi = tau; else lo = tau;
                    double step;
                    bool model;
                    nt = secular_step(f, dpsi, dphi, tau, lo, hi, deli, deli1, last, &step, &model);
                    if (hi - lo <= 4.0 * TD_EPS * fmax(fabs(lo), fabs(hi)) ||
                        (model && fabs(step) <= 1e-12 * fabs(tau)))
                        stop = 1;
                }
            }
            stop = __shfl_sync(FULL, stop, 0, G);
            nt = __shfl_sync(FULL, nt, 0, G);
            if (dfrun) {
                tau = nt;
                itdf++;
                if (stop) dfrun = false;
            }
        }
        *df_iters = itdf;
    }
    lo = lo0;
    hi = hi0;

    // ---- FP64 iterations (as secular_root_warp) ---------------------------
    bool frun = run;
    int it = 0;
    for (int t = 1; t <= TD_SECULAR_MAXIT; t++) {
        if (!__any_sync(FULL, frun)) break;
        double s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0;
        const int ie = frun ? i : -1, ke = frun ? K : 0;
        for (int j = gl; j <= ie; j += G) {
            double q = td_recip((d[j] - dorg) - tau);
            double tt = w[j] * q;
            s1 += tt; s2 += tt * q;
        }
        for (int j = i + 1 + gl; j < ke; j += G) {
            double q = td_recip((d[j] - dorg) - tau);
            double tt = w[j] * q;
            s3 += tt; s4 += tt * q;
        }
        const double psi = grp_sum_d<G>(s1), dpsi = grp_sum_d<G>(s2);
        const double phi = grp_sum_d<G>(s3), dphi = grp_sum_d<G>(s4);
        int stop = 0;
        double nt = tau;
        if (frun && gl == 0) {
            const double f = 1.0 + psi + phi;
            const double err = 8.0 * TD_EPS * (1.0 + fabs(psi) + fabs(phi) + fabs(tau) * (dpsi + dphi));
            if (fabs(f) <= err) {
                stop = 1;
            } else {
                if (f > 0.0) hi = tau; else lo = tau;
                if (hi - lo <= 4.0 * TD_EPS * fmax(fabs(lo), fabs(hi))) {
                    stop = 1;
                } else {
                    double step;
                    bool model;
                    nt = secular_step(f, dpsi, dphi, tau, lo, hi, deli, deli1, last, &step, &model);
                    if (nt == tau) stop = 1;
                    else if (model && fabs(step) <= 1e-9 * fabs(tau)) stop = 2;
                }
            }
        }
        stop = __shfl_sync(FULL, stop, 0, G);
        nt = __shfl_sync(FULL, nt, 0, G);
        if (frun) {
            it = t;
            if (stop == 1) frun = false;
            else {
                tau = nt;
                if (stop == 2) frun = false;
            }
        }
    }
    if (frun) it = TD_SECULAR_MAXIT + 1;   // not converged
    if (run) {
        *lam = dorg + tau;
        if (last) { *gam = tau; *mu = 0.0; }
        else if (org == i) { *gam = tau; *mu = (d[i + 1] - d[i]) - tau; }
        else { *mu = -tau; *gam = (d[i + 1] - d[i]) + tau; }
        *iters = it;
    } else if (act) {
        *lam = d[0] + w[0]; *gam = w[0]; *mu = 0.0; *iters = 0;
    }
}

// Merges of at most this many poles take the grouped form (G = 4 up to 64, 8
// up to 128, 16 up to 256).
#define TD_SECULAR_GRP_MAXK 256

template <int G>
__global__ void k_secular_grp(const MergeDesc* M, int nmerge, int rows, LevelWS ws, int* status)
{
    const int tg = blockIdx.x * blockDim.x + threadIdx.x;
    if (((tg & ~31) / G) >= rows) return;   // the warp's first root: whole warps leave
    const int gl = threadIdx.x & (G - 1);
    const int r = tg / G;
    int g0 = 0, i = 0, K = 0;
    bool act = false;
    if (r < rows) {
        const int m = td_find_merge(M, nmerge, r);
        if (m >= 0) {
            g0 = M[m].g0;
            i = r - g0;
            K = ws.K[m];
            act = i < K;
        }
    }
    if (!act) { g0 = 0; i = 0; K = 0; }
    double lam = 0.0, gam = 0.0, mu = 0.0;
    int it, itdf;
    secular_root_group<G>(ws.dK + g0, ws.wK + g0, K, i, act, gl, &lam, &gam, &mu, &it, &itdf,
                          ws.dhK + g0, ws.dlK + g0, ws.wfK + g0, ws.wlK + g0);
    if (act && gl == 0) {
        ws.lamK[g0 + i] = lam;
        ws.gamK[g0 + i] = gam;
        ws.muK[g0 + i] = mu;
        if (it > TD_SECULAR_MAXIT) atomicOr(status, TD_STATUS_NOTCONV);
        atomicAdd((unsigned long long*)(status + TD_STATUS_SECULAR_TERMS),
                  (unsigned long long)(min(it, TD_SECULAR_MAXIT) + (i == K - 1 ? 1 : 0)) *
                      (unsigned long long)K);
        atomicAdd((unsigned long long*)(status + TD_STATUS_SECULAR_DFTERMS),
                  (unsigned long long)itdf * (unsigned long long)K);
    }
}

__global__ void k_secular(const MergeDesc* M, int nmerge, int rows, LevelWS ws, int* status)
{
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= rows) return;
    const int m = td_find_merge(M, nmerge, gw);
    if (m < 0) return;
    const int g0 = M[m].g0;
    const int i = gw - g0;
    const int K = ws.K[m];
    if (i >= K) return;
    double lam, gam, mu;
    int it, itdf;
    secular_root_warp(ws.dK + g0, ws.wK + g0, K, i, lane, &lam, &gam, &mu, &it, &itdf,
                      ws.dhK + g0, ws.dlK + g0, ws.wfK + g0, ws.wlK + g0);
    if (lane == 0) {
        ws.lamK[g0 + i] = lam;
        ws.gamK[g0 + i] = gam;
        ws.muK[g0 + i] = mu;
        if (it > TD_SECULAR_MAXIT) atomicOr(status, TD_STATUS_NOTCONV);
        // work count: K FP64 terms per FP64 evaluation (the last root's FP64
        // bracket sum included), K double-float terms per double-float one (the
        // FP32 midpoint value is not counted)
        atomicAdd((unsigned long long*)(status + TD_STATUS_SECULAR_TERMS),
                  (unsigned long long)(min(it, TD_SECULAR_MAXIT) + (i == K - 1 ? 1 : 0)) *
                      (unsigned long long)K);
        atomicAdd((unsigned long long*)(status + TD_STATUS_SECULAR_DFTERMS),
                  (unsigned long long)itdf * (unsigned long long)K);
    }
}

// Lanes per root: the smallest group the merge size allows (4 up to 64 poles, 8
// up to 128, 16 up to 256, else a warp), widened while the launch would have
// fewer than 16 warps per SM (fewer roots per warp then hide more latency).
static int secular_group(int nmax, int rows)
{
    int g = nmax <= 64 ? 4 : nmax <= 128 ? 8 : nmax <= TD_SECULAR_GRP_MAXK ? 16 : 32;
    while (g < 32 && (long long)rows * g / 32 < 16LL * td_sm_count()) g *= 2;
    return g;
}

void td_launch_secular(const MergeDesc* M, int nmerge, int rows, int nmax, const LevelWS& ws,
                       int* status, cudaStream_t st)
{
    if (rows <= 0) return;
    td_prof_begin(st);
    switch (secular_group(nmax, rows)) {
    case 4: k_secular_grp<4><<<td_cdiv(rows, 64), 256, 0, st>>>(M, nmerge, rows, ws, status); break;
    case 8: k_secular_grp<8><<<td_cdiv(rows, 32), 256, 0, st>>>(M, nmerge, rows, ws, status); break;
    case 16: k_secular_grp<16><<<td_cdiv(rows, 16), 256, 0, st>>>(M, nmerge, rows, ws, status); break;
    default: k_secular<<<td_cdiv(rows, 8), 256, 0, st>>>(M, nmerge, rows, ws, status); break;
    }
    td_prof_end(st, "k_secular");
}

// ---------------------------------------------------------------------------
// Loewner (eq. ev_z with 1/rho): uhat_i^2 = gamma_i/rho prod_{j != i}
// (lambda_j - d_i)/(d_j - d_i), each lambda_j - d_i by Remark 1; sign of z_i.
// One warp per i; lane-strided partial products, then a shuffle product.
// ---------------------------------------------------------------------------
__global__ void k_lowner(const MergeDesc* M, int nmerge, int rows, LevelWS ws)
{
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= rows) return;
    const int m = td_find_merge(M, nmerge, gw);
    if (m < 0) return;
    const int g0 = M[m].g0;
    const int i = gw - g0;
    const int K = ws.K[m];
    if (i >= K) return;
    const double* d = ws.dK + g0;
    const double* gam = ws.gamK + g0;
    const double* mu = ws.muK + g0;
    const double di = d[i];
    // Numerators and denominators multiplied separately (one divide per lane
    // instead of one per term), each brought back to [1, 2) every 4 factors with
    // its power of two kept in an integer: a factor of the scaled matrix is at
    // most 8 in magnitude, and 4 of them stay inside the FP64 range unless pole
    // gaps fall below 1e-75.
    // lambda_j - d_i by Remark 1: (d_j+1 - d_i) - mu_j for j < i, (d_j - d_i) +
    // gamma_j for j > i (reusing the denominator): two loops, so that no term
    // evaluates both forms (a select of the two cost the FP64 pipe both)
    double pn = 1.0, pd = 1.0;
    int ex = 0, cnt = 0;
    for (int j = lane; j < i; j += 32) {
        pn *= (d[j + 1] - di) - mu[j];
        pd *= d[j] - di;
        if (++cnt == 4) {
            cnt = 0;
            pn = td_renorm(pn, &ex, 1);
            pd = td_renorm(pd, &ex, -1);
        }
    }
    for (int j = i + 1 + lane; j < K; j += 32) {
        const double den = d[j] - di;
        pn *= den + gam[j];
        pd *= den;
        if (++cnt == 4) {
            cnt = 0;
            pn = td_renorm(pn, &ex, 1);
            pd = td_renorm(pd, &ex, -1);
        }
    }
    pn = td_renorm(pn, &ex, 1);
    pd = td_renorm(pd, &ex, -1);
    double p = pn / pd;   // in (1/2, 2)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double q = __shfl_xor_sync(0xffffffffu, p, o);
        const int eq = __shfl_xor_sync(0xffffffffu, ex, o);
        p = td_renorm(p * q, &ex, 1);
        ex += eq;
    }
    if (lane == 0) {
        double u = sqrt(scalbn(gam[i] / ws.rho[m] * p, ex));
        const double us = copysign(u, ws.zK[g0 + i]);
        ws.uhat[g0 + i] = us;
        const float uf = __double2float_rn(us);
        ws.ufK[g0 + i] = uf;
        ws.ulK[g0 + i] = __double2float_rn(us - (double)uf);
    }
}

// ---------------------------------------------------------------------------
// Cauchy-like eigenvector matrix (eq. Ev-Q): one CTA per column j.
//   t_k = uhat_k / (d_k - lambda_j), v_j = 1/sqrt(sum t_k^2), Qhat[k, j] = t_k v_j.
// The column is kept in shared memory when it fits, else recomputed.
// ---------------------------------------------------------------------------
#define CAUCHY_NT 256
template <bool SMEM>
__global__ void __launch_bounds__(CAUCHY_NT) k_cauchy(const MergeDesc* M, int nmerge, int rows,
                                                      LevelWS ws, int write_qhat)
{
    extern __shared__ double col[];
    __shared__ double red[32];
    const int gcol = blockIdx.x;
    if (gcol >= rows) return;
    const int m = td_find_merge(M, nmerge, gcol);
    if (m < 0) return;
    const MergeDesc& md = M[m];
    const int g0 = md.g0;
    const int j = gcol - g0;
    const int K = ws.K[m];
    if (j >= K) return;
    const double* d = ws.dK + g0;
    const double* gam = ws.gamK + g0;
    const double* mu = ws.muK + g0;
    const double* uh = ws.uhat + g0;
    // write_qhat: 0 v only; 1 rows in secular order; 2 rows in the order of the
    // update product (gemmCol), so the product reads Qhat contiguously.
    const int* perm = (write_qhat == 2) ? ws.gemmCol + g0 : nullptr;
    // d_k - lambda_j (Remark 1) with the column's poles and offsets held in
    // registers: (d_k - d_j) - gamma_j for k <= j, (d_k - d_j+1) + mu_j above
    const double dj = d[j], ngj = -gam[j];
    const double dj1 = (j + 1 < K) ? d[j + 1] : 0.0, mj = mu[j];
    auto term = [&](int k) {
        const bool below = (k <= j);
        return uh[k] * td_recip((d[k] - (below ? dj : dj1)) + (below ? ngj : mj));
    };
    double acc = 0.0;
    for (int p = threadIdx.x; p < K; p += blockDim.x) {
        const double t = term(perm ? perm[p] : p);
        if (SMEM) col[p] = t;
        acc += t * t;
    }
    // warp sums, then the warps' partial sums and the FP64 square root and
    // divide by one thread (every thread repeating them cost the 1/64-rate FP64
    // pipe a sizeable share of a small column)
    acc = td_warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    __shared__ double s_vj;
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) acc += red[w];
        s_vj = 1.0 / sqrt(acc);
        ws.vv[g0 + j] = s_vj;
    }
    __syncthreads();
    const double vj = s_vj;
    if (!write_qhat) return;
    // leading dimension: n in the product order used by the dense update (its
    // launches can then be sized without knowing K), K in secular order
    double* out = md.qhat + (int64_t)j * (write_qhat == 2 ? md.n : K);
    for (int p = threadIdx.x; p < K; p += blockDim.x) {
        const double t = SMEM ? col[p] : term(perm ? perm[p] : p);
        out[p] = t * vj;
    }
}

// ---------------------------------------------------------------------------
// The Cauchy-like matrix in double-float, for solves whose products are split
// precision (42-bit slices): the column norms v and the entries of Qhat are
// formed from FP32 pairs on the FP32 pipe, 64x the FP64 rate on this part
// (the FP64 form above keeps that pipe ~85 % busy).  Pole differences are
// exact inputs to it: each pole is held as an exact FP32 triple (dhK + dlK +
// dxK = dK), so d_k - d_j comes out of TwoSums of the parts with a relative
// error of about 2^-47 however close the poles; the Remark 1 offset
// (-gamma_j or mu_j) has the same sign, so d_k - lambda_j keeps that relative
// accuracy, and the reciprocal (one Newton step from the FP32 estimate), the
// product with uhat and the squares keep entries and norms within ~2^-44 --
// below the 2^-42 of the split products that use them.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void df_fast_two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

// d_k - p for exact triples (kh + km + kx, ph + pm + px) as a double-float.
__device__ __forceinline__ void df_pole_diff(float kh, float km, float kx, float ph, float pm,
                                             float px, float& rh, float& rl)
{
    float s1, e1, s2, e2, t, u;
    df_two_sum(kh, -ph, s1, e1);
    df_two_sum(km, -pm, s2, e2);
    const float s3 = __fsub_rn(kx, px);
    df_two_sum(s1, s2, t, u);
    const float lo = __fadd_rn(__fadd_rn(__fadd_rn(e1, e2), s3), u);
    df_two_sum(t, lo, rh, rl);
}

// uhat_k / (d_k - lambda_j) as a double-float (th, tl).
__device__ __forceinline__ void df_cauchy_entry(float kh, float km, float kx, float ph, float pm,
                                                float px, float oh, float ol, float uh, float ul,
                                                float& th, float& tl)
{
    float Ph, Pl, a, b, Dh, Dl;
    df_pole_diff(kh, km, kx, ph, pm, px, Ph, Pl);
    df_two_sum(Ph, oh, a, b);                       // same signs: no cancellation
    b = __fadd_rn(b, __fadd_rn(Pl, ol));
    df_fast_two_sum(a, b, Dh, Dl);
    const float q0 = td_rcp_f32(Dh);
    float r = fmaf(-Dh, q0, 1.0f);
    r = fmaf(-Dl, q0, r);
    const float ql = __fmul_rn(q0, r);
    th = __fmul_rn(uh, q0);
    tl = __fadd_rn(fmaf(uh, q0, -th), fmaf(uh, ql, __fmul_rn(ul, q0)));
}

// An FP32 value as FP64 by assembling the bit pattern (sign, rebiased exponent,
// mantissa) with integer operations: exact for normal values, like a
// conversion, but off the 1/64-rate FP64 pipe that conversions issue on.
// Subnormal FP32 values (below 1.2e-38) are taken as zero.
__device__ __forceinline__ double td_f2d_bits(float x)
{
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned long long ee = (e == 0xffu) ? 0x7ffull : (unsigned long long)(e + 896u);
    const unsigned long long b = ((unsigned long long)(u >> 31) << 63) | (ee << 52) |
                                 ((unsigned long long)(u & 0x7fffffu) << 29);
    return e == 0u ? 0.0 : __longlong_as_double(b);
}

template <bool SMEM>
__global__ void __launch_bounds__(CAUCHY_NT) k_cauchy_df(const MergeDesc* M, int nmerge, int rows,
                                                         LevelWS ws, int write_qhat)
{
    extern __shared__ float2 colf[];
    const int gcol = blockIdx.x;
    if (gcol >= rows) return;
    const int m = td_find_merge(M, nmerge, gcol);
    if (m < 0) return;
    const MergeDesc& md = M[m];
    const int g0 = md.g0;
    const int j = gcol - g0;
    const int K = ws.K[m];
    if (j >= K) return;
    const float* dh = ws.dhK + g0;
    const float* dm = ws.dlK + g0;
    const float* dx = ws.dxK + g0;
    const float* uf = ws.ufK + g0;
    const float* ul = ws.ulK + g0;
    const int* perm = (write_qhat == 2) ? ws.gemmCol + g0 : nullptr;
    // the column's poles (j and j+1) and Remark 1 offsets as FP32 parts
    const float pjh = dh[j], pjm = dm[j], pjx = dx[j];
    const bool hasn = j + 1 < K;
    const float pnh = hasn ? dh[j + 1] : 0.0f, pnm = hasn ? dm[j + 1] : 0.0f,
                pnx = hasn ? dx[j + 1] : 0.0f;
    // the offsets' FP32 pairs by one thread (FP64 conversions issue on the
    // 1/64-rate pipe; repeated by every thread they outweighed a small column)
    __shared__ float s_off[4];
    if (threadIdx.x == 0) {
        const double ng = -ws.gamK[g0 + j], mj = ws.muK[g0 + j];
        const float a = __double2float_rn(ng), b = __double2float_rn(mj);
        s_off[0] = a;
        s_off[1] = __double2float_rn(ng - (double)a);
        s_off[2] = b;
        s_off[3] = __double2float_rn(mj - (double)b);
    }
    __syncthreads();
    const float ngh = s_off[0], ngl = s_off[1], mjh = s_off[2], mjl = s_off[3];
    auto term = [&](int k, float& th, float& tl) {
        const bool below = (k <= j);
        df_cauchy_entry(dh[k], dm[k], dx[k], below ? pjh : pnh, below ? pjm : pnm,
                        below ? pjx : pnx, below ? ngh : mjh, below ? ngl : mjl, uf[k], ul[k],
                        th, tl);
    };
    float Ah = 0.0f, Al = 0.0f;
    for (int p = threadIdx.x; p < K; p += blockDim.x) {
        float th, tl;
        term(perm ? perm[p] : p, th, tl);
        if (SMEM) colf[p] = make_float2(th, tl);
        // (th + tl)^2 to the double-float sum, renormalised every term (a low
        // part left to grow would carry a rounding error per term)
        const float sh = __fmul_rn(th, th);
        const float sl = fmaf(2.0f * th, tl, fmaf(th, th, -sh));
        float s, e;
        df_two_sum(Ah, sh, s, e);
        df_fast_two_sum(s, __fadd_rn(Al, __fadd_rn(e, sl)), Ah, Al);
    }
    // block sum in double-float (FP32 shuffles and TwoSums); one thread turns it
    // into FP64 (an FP64 sum over all threads cost more than a small column)
    df_warp_sum(Ah, Al);
    __shared__ float2 s_part[CAUCHY_NT / 32];
    __shared__ float s_vf[2];
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = make_float2(Ah, Al);
    __syncthreads();
    if (threadIdx.x == 0) {
        float h = s_part[0].x, l = s_part[0].y;
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
            float t, e;
            df_two_sum(h, s_part[w].x, t, e);
            df_fast_two_sum(t, __fadd_rn(l, __fadd_rn(e, s_part[w].y)), h, l);
        }
        const double vj = 1.0 / sqrt(td_f2d_bits(h) + td_f2d_bits(l));
        ws.vv[g0 + j] = vj;
        s_vf[0] = __double2float_rn(vj);
        s_vf[1] = __double2float_rn(vj - (double)s_vf[0]);
    }
    __syncthreads();
    if (!write_qhat) return;
    const float vh = s_vf[0], vl = s_vf[1];
    double* out = md.qhat + (int64_t)j * (write_qhat == 2 ? md.n : K);
    for (int p = threadIdx.x; p < K; p += blockDim.x) {
        float th, tl;
        if (SMEM) { const float2 t2 = colf[p]; th = t2.x; tl = t2.y; }
        else term(perm ? perm[p] : p, th, tl);
        const float ph = __fmul_rn(th, vh);
        const float pl = __fadd_rn(fmaf(th, vh, -ph), fmaf(th, vl, __fmul_rn(tl, vh)));
        out[p] = td_f2d_bits(ph) + td_f2d_bits(pl);
    }
}

#define CAUCHY_SMEM_MAX 200000
static void launch_cauchy(const MergeDesc* M, int nmerge, int rows, int kmax, const LevelWS& ws,
                          int write_qhat, cudaStream_t st, bool df = false)
{
    size_t sm = (size_t)kmax * sizeof(double);
    // one CTA per column, as many threads as the longest column needs (at most
    // CAUCHY_NT): idle warps of small columns only added reduction work
    const int nt = std::min(CAUCHY_NT, std::max(32, td_cdiv(kmax, 32) * 32));
    if (df) {
        // double-float form (the FP32 parts of the poles and of uhat are in ws)
        if (sm <= CAUCHY_SMEM_MAX) {
            td_smem_attr((const void*)k_cauchy_df<true>, CAUCHY_SMEM_MAX);
            td_prof_begin(st); k_cauchy_df<true><<<rows, nt, sm, st>>>(M, nmerge, rows, ws, write_qhat); td_prof_end(st, "k_cauchy");
        } else {
            td_prof_begin(st); k_cauchy_df<false><<<rows, nt, 0, st>>>(M, nmerge, rows, ws, write_qhat); td_prof_end(st, "k_cauchy");
        }
        return;
    }
    if (sm <= CAUCHY_SMEM_MAX) {
        td_smem_attr((const void*)k_cauchy<true>, CAUCHY_SMEM_MAX);
        td_prof_begin(st); k_cauchy<true><<<rows, nt, sm, st>>>(M, nmerge, rows, ws, write_qhat); td_prof_end(st, "k_cauchy");
    } else {
        td_prof_begin(st); k_cauchy<false><<<rows, nt, 0, st>>>(M, nmerge, rows, ws, write_qhat); td_prof_end(st, "k_cauchy");
    }
}

void td_launch_cauchy(const MergeDesc* M, int nmerge, int rows, int kmax, const LevelWS& ws,
                      int write_qhat, cudaStream_t st)
{
    if (rows <= 0) return;
    launch_cauchy(M, nmerge, rows, kmax, ws, write_qhat, st);
}

void td_launch_lowner_cauchy(const MergeDesc* M, int nmerge, int rows, int kmax, const LevelWS& ws,
                             int write_qhat, cudaStream_t st, bool df)
{
    if (rows <= 0) return;
    td_prof_begin(st); k_lowner<<<td_cdiv(rows, 8), 256, 0, st>>>(M, nmerge, rows, ws); td_prof_end(st, "k_lowner");
    launch_cauchy(M, nmerge, rows, kmax, ws, write_qhat, st, df);
}

// ---------------------------------------------------------------------------
// Final ordering: new eigenvalues lambda (ascending) and deflated d merged into
// ascending order, new ones first on ties (stable).  Positions feed the GEMM
// epilogue and the deflated-column copy.
//
// When the deflated poles are ascending (no rotation moved one past another)
// each position is a binary search, one CTA per merge (k_order).  Otherwise
// k_order only flags the merge and the position of each of the n values (the
// K new ones, then the n - K deflated ones) is its rank in the order (value,
// then that index), counted in parallel by k_order_count and written by
// k_order_place.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PREP_NT) k_order(const MergeDesc* M, LevelWS ws)
{
    __shared__ double red[32];
    MergeDesc md = M[blockIdx.x];
    const int n = md.n, g0 = md.g0;
    const int K = ws.K[blockIdx.x];
    const int nd = n - K;
    const int* dfl = ws.deflIdx + g0;
    const double* ds = ws.dsort + g0;
    const double* lk = ws.lamK + g0;
    // are the deflated values ascending?
    double bad = 0.0;
    for (int l = threadIdx.x; l + 1 < nd; l += blockDim.x)
        if (!(ds[dfl[l + 1]] >= ds[dfl[l]])) bad = 1.0;
    const bool sorted = blk_max(bad, red) == 0.0;
    if (threadIdx.x == 0) ws.unsorted[blockIdx.x] = sorted ? 0 : 1;
    if (!sorted) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) ws.ordr[g0 + i] = 0;
        return;
    }
    const double scale = md.scale_ptr ? *md.scale_ptr : 1.0;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double v = lk[k];
        int lo = 0, hi = nd;   // count of deflated < v
        while (lo < hi) { int mid = (lo + hi) >> 1; if (ds[dfl[mid]] < v) lo = mid + 1; else hi = mid; }
        ws.posNew[g0 + k] = k + lo;
        md.lam_out[k + lo] = v * scale;
    }
    for (int l = threadIdx.x; l < nd; l += blockDim.x) {
        double v = ds[dfl[l]];
        int lo = 0, hi = K;   // count of new <= v
        while (lo < hi) { int mid = (lo + hi) >> 1; if (lk[mid] <= v) lo = mid + 1; else hi = mid; }
        ws.posDefl[g0 + l] = l + lo;
        md.lam_out[l + lo] = v * scale;
    }
}

#define ORD_CH 2048

__device__ __forceinline__ double order_value(const LevelWS& ws, int g0, int K, int i)
{
    return i < K ? ws.lamK[g0 + i] : ws.dsort[g0 + ws.deflIdx[g0 + i - K]];
}

// Grid: (merge, 256-value tile, ORD_CH-value chunk).  Each thread counts the
// values of the chunk that precede its own value.
__global__ void __launch_bounds__(256) k_order_count(const MergeDesc* M, LevelWS ws)
{
    __shared__ double sv[ORD_CH];
    if (!ws.unsorted[blockIdx.x]) return;
    const int n = M[blockIdx.x].n, g0 = M[blockIdx.x].g0;
    const int K = ws.K[blockIdx.x];
    const int i0 = blockIdx.y * 256, j0 = blockIdx.z * ORD_CH;
    if (i0 >= n || j0 >= n) return;
    const int jn = min(ORD_CH, n - j0);
    for (int j = threadIdx.x; j < jn; j += 256) sv[j] = order_value(ws, g0, K, j0 + j);
    __syncthreads();
    const int i = i0 + threadIdx.x;
    if (i >= n) return;
    const double v = order_value(ws, g0, K, i);
    int c = 0;
    // values of the chunk strictly before i in index order win ties
    const int jt = min(max(i - j0, 0), jn);
    for (int j = 0; j < jt; j++) c += (sv[j] <= v);
    for (int j = jt; j < jn; j++) c += (sv[j] < v);
    atomicAdd(&ws.ordr[g0 + i], c);
}

// Grid: (merge, 256-value tile).
__global__ void __launch_bounds__(256) k_order_place(const MergeDesc* M, LevelWS ws)
{
    if (!ws.unsorted[blockIdx.x]) return;
    const MergeDesc& md = M[blockIdx.x];
    const int n = md.n, g0 = md.g0;
    const int K = ws.K[blockIdx.x];
    const int i = blockIdx.y * 256 + threadIdx.x;
    if (i >= n) return;
    const double scale = md.scale_ptr ? *md.scale_ptr : 1.0;
    const int pos = min(max(ws.ordr[g0 + i], 0), n - 1);
    if (i < K) ws.posNew[g0 + i] = pos;
    else ws.posDefl[g0 + i - K] = pos;
    md.lam_out[pos] = order_value(ws, g0, K, i) * scale;
}

// Grid: (merge, 256-row tile, 32-column tile).
__global__ void k_copy_defl(const MergeDesc* M, LevelWS ws)
{
    MergeDesc md = M[blockIdx.x];
    const int n = md.n, g0 = md.g0;
    const int nd = n - ws.K[blockIdx.x];
    const int rt = blockIdx.y, ct = blockIdx.z;
    if (ct * 32 >= nd) return;
    const int r = rt * 256 + threadIdx.x;
    if (r >= n) return;
    for (int cc = 0; cc < 32; cc++) {
        int l = ct * 32 + cc;
        if (l >= nd) break;
        md.qout[(int64_t)ws.posDefl[g0 + l] * n + r] = md.W[(int64_t)ws.deflIdx[g0 + l] * n + r];
    }
}

void td_launch_finish(const MergeDesc* M, int nmerge, int nmax, const LevelWS& ws, cudaStream_t st)
{
    dim3 g(nmerge, td_cdiv(nmax, 256), td_cdiv(nmax, 32));
    td_prof_begin(st); k_copy_defl<<<g, 256, 0, st>>>(M, ws); td_prof_end(st, "k_copy_defl");
}

// ---------------------------------------------------------------------------
// Dense update (plain DC): C = W[:, surv] * Qhat, C column k written to the
// output column posNew[k].  FP64 on the CUDA cores: a BM x BN x 16 shared-
// memory tile, (BM/16) x (BN/16) outputs per thread (rows tx + 16 a, cols
// ty + 16 b).  On this part FP64 FMA issue (~1.2 TFLOP/s measured) is at least
// as fast as the FP64 mma.sync path (~1.05 TFLOP/s measured), so the SIMT form
// is used.  Tile shapes are chosen per level by the autotuner in the host code;
// toff[m] is the first tile of merge m for the chosen shape (prefix sums).
// ---------------------------------------------------------------------------
template <int BM, int BN>
__global__ void __launch_bounds__(256) k_gemm_f64(const MergeDesc* M, const int* toff, int nmerge,
                                                 LevelWS ws)
{
    constexpr int TA = BM / 16, TB = BN / 16;
    __shared__ double As[TD_GEMM_BK][BM];
    __shared__ double Bs[TD_GEMM_BK][BN + 1];
    int lo = 0, hi = nmerge - 1;
    const int bid = blockIdx.x;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (toff[mid] <= bid) lo = mid; else hi = mid - 1;
    }
    const MergeDesc& md = M[lo];
    const int m = lo;
    const int n = md.n, g0 = md.g0;
    const int K = ws.K[m];
    const int tiles_m = td_cdiv(n, BM);
    const int local = bid - toff[lo];
    const int tm = local % tiles_m, tn = local / tiles_m;
    const int row0 = tm * BM, col0 = tn * BN;
    if (col0 >= K || K == 0) return;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int* wcol = ws.gemmW + g0;
    const double* W = md.W;
    const double* B = md.qhat;   // rows already in product order
    // Block structure of diag(Q1, Q2) after deflation: child-1 rows see only
    // product positions [0, K1 + Km), child-2 rows only [K1, K).
    const int K1 = ws.kgrp[2 * m], Km = ws.kgrp[2 * m + 1];
    const int kbeg = (row0 >= md.n1) ? K1 : 0;
    const int kend = (row0 + BM <= md.n1) ? K1 + Km : K;
    double acc[TA][TB];
#pragma unroll
    for (int a = 0; a < TA; a++)
#pragma unroll
        for (int b = 0; b < TB; b++) acc[a][b] = 0.0;

    for (int k0 = kbeg; k0 < kend; k0 += TD_GEMM_BK) {
#pragma unroll
        for (int q = 0; q < TA; q++) {
            const int idx = threadIdx.x + 256 * q;
            const int kk = idx / BM, r = idx % BM;
            const int k = k0 + kk, row = row0 + r;
            As[kk][r] = (k < kend && row < n) ? W[(int64_t)wcol[k] * n + row] : 0.0;
        }
#pragma unroll
        for (int q = 0; q < TB; q++) {
            const int idx = threadIdx.x + 256 * q;
            const int kb = idx & 15, c = idx >> 4;
            const int kg = k0 + kb, cg = col0 + c;
            Bs[kb][c] = (kg < kend && cg < K) ? B[(int64_t)cg * n + kg] : 0.0;   // Qhat: ld n
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TD_GEMM_BK; kk++) {
            double av[TA], bv[TB];
#pragma unroll
            for (int a = 0; a < TA; a++) av[a] = As[kk][tx + 16 * a];
#pragma unroll
            for (int b = 0; b < TB; b++) bv[b] = Bs[kk][ty + 16 * b];
#pragma unroll
            for (int a = 0; a < TA; a++)
#pragma unroll
                for (int b = 0; b < TB; b++) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int b = 0; b < TB; b++) {
        const int c = col0 + ty + 16 * b;
        if (c >= K) continue;
        double* out = md.qout + (int64_t)ws.posNew[g0 + c] * n;
#pragma unroll
        for (int a = 0; a < TA; a++) {
            const int r = row0 + tx + 16 * a;
            if (r < n) out[r] = acc[a][b];
        }
    }
}

void td_gemm_tiles(int variant, int n, int* bm, int* bn)
{
    static const int shapes[TD_GEMM_VARIANTS][2] = {{64, 64}, {32, 32}, {128, 64}, {64, 32}};
    *bm = shapes[variant][0];
    *bn = shapes[variant][1];
    (void)n;
}

void td_launch_update_dense(const MergeDesc* M, const int* toff, int nmerge, int total_tiles,
                            int variant, const LevelWS& ws, cudaStream_t st)
{
    if (total_tiles <= 0) return;
    td_prof_begin(st);
    switch (variant) {
    case 1: k_gemm_f64<32, 32><<<total_tiles, 256, 0, st>>>(M, toff, nmerge, ws); break;
    case 2: k_gemm_f64<128, 64><<<total_tiles, 256, 0, st>>>(M, toff, nmerge, ws); break;
    case 3: k_gemm_f64<64, 32><<<total_tiles, 256, 0, st>>>(M, toff, nmerge, ws); break;
    default: k_gemm_f64<64, 64><<<total_tiles, 256, 0, st>>>(M, toff, nmerge, ws); break;
    }
    td_prof_end(st, "k_gemm_f64");
}

// Order kernel launcher (separate so the HSS path can reuse it).
void td_launch_order(const MergeDesc* M, int nmerge, int nmax, const LevelWS& ws, cudaStream_t st)
{
    td_prof_begin(st); k_order<<<nmerge, PREP_NT, 0, st>>>(M, ws); td_prof_end(st, "k_order");
    dim3 gc(nmerge, td_cdiv(nmax, 256), td_cdiv(nmax, ORD_CH));
    td_prof_begin(st); k_order_count<<<gc, 256, 0, st>>>(M, ws); td_prof_end(st, "k_order_count");
    dim3 gp(nmerge, td_cdiv(nmax, 256));
    td_prof_begin(st); k_order_place<<<gp, 256, 0, st>>>(M, ws); td_prof_end(st, "k_order_place");
}

// Stage entry points: one rank-one problem of size K placed as merge 0.
__global__ void k_stage_init(LevelWS ws, int K, double rho)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) { ws.K[0] = K; ws.rho[0] = rho; ws.nrot[0] = 0; }
    if (i < K) {
        double z = ws.zK[i];
        const double w = rho * z * z, di = ws.dK[i];
        ws.wK[i] = w;
        const float dh = __double2float_rn(di);
        ws.dhK[i] = dh;
        const double r1 = di - (double)dh;
        const float dm = __double2float_rn(r1);
        ws.dlK[i] = dm;
        ws.dxK[i] = __double2float_rn(r1 - (double)dm);
        const float wh = __double2float_rn(w);
        ws.wfK[i] = wh;
        ws.wlK[i] = __double2float_rn(w - (double)wh);
    }
}

void td_launch_stage_init(const LevelWS& ws, int K, double rho, cudaStream_t st)
{
    td_prof_begin(st); k_stage_init<<<td_cdiv(std::max(K, 1), 256), 256, 0, st>>>(ws, K, rho); td_prof_end(st, "k_stage_init");
}

// ---------------------------------------------------------------------------
// Secular roots without any allocation (tdeig_secular_noalloc in tdeig.h).
//
// Some callers cannot allocate device memory at the moment they need the
// roots: code that has handed all free device memory to its own pool
// allocator (a cudaMalloc there fails or fragments the pool), and code on a
// latency-bound path where cudaMalloc's implicit device synchronisation is not
// acceptable.  This variant of the secular stage keeps its scratch -- the
// weights rho z_j^2 in FP64 and as FP32 pairs, the FP32 pair of each pole, and
// a status word -- in the file-scope array below, which every GPU that loads the
// library holds until the process exits.  With that scratch it runs the same
// per-root iteration as k_secular (FP32 midpoint value, two-pole start), so
// its roots are those of tdeig_secular bit for bit.
//
// Host code cannot use the array's name as a device address: it is a host-side
// stand-in.  The first call on each device (with that device current) looks
// the device address up with cudaGetSymbolAddress and caches it; make that
// first call before any stream capture.  All calls share the array, so calls
// whose work overlaps on the GPU (other streams, other host threads) race.
// ---------------------------------------------------------------------------
// layout in doubles: w [0, MAX_K); then MAX_K floats each of wf, wl, dh, dl
// (2 MAX_K doubles); then the status word
#define TD_NOALLOC_F32 TDEIG_NOALLOC_MAX_K
#define TD_NOALLOC_STATUS (3 * TDEIG_NOALLOC_MAX_K)
#define TD_NOALLOC_SLOTS (TD_NOALLOC_STATUS + 32)
static __device__ __align__(256) double td_noalloc_scratch[TD_NOALLOC_SLOTS];

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[TD_NOALLOC_MAX_DEVICES];

// The weights and FP32 copies of one problem (as k_stage_init forms them for
// tdeig_secular), and the status word cleared for this call.
__global__ void k_noalloc_weights(const double* d, const double* z, double rho, int K, double* w,
                                  float* wf, float* wl, float* dh, float* dl, int* status)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *status = 0;   // clear the status word the previous call left in the array
    if (i < K) {
        const double wi = rho * z[i] * z[i], di = d[i];
        w[i] = wi;
        const float h = __double2float_rn(di);
        dh[i] = h;
        dl[i] = __double2float_rn(di - (double)h);
        const float wh = __double2float_rn(wi);
        wf[i] = wh;
        wl[i] = __double2float_rn(wi - (double)wh);
    }
}

__global__ void k_secular_noalloc(const double* d, const double* w, const float* wf, const float* wl,
                                  const float* dh, const float* dl, int K, int* status,
                                  double* lam, double* gam, double* mu)
{
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= K) return;
    double l, g, m;
    int it, itdf;
    secular_root_warp(d, w, K, i, lane, &l, &g, &m, &it, &itdf, dh, dl, wf, wl);
    if (lane == 0) {
        lam[i] = l;
        gam[i] = g;
        mu[i] = m;
        if (it > TD_SECULAR_MAXIT) atomicOr(status, TD_STATUS_NOTCONV);
    }
}

// The grouped form for K <= TD_SECULAR_GRP_MAXK, chosen as tdeig_secular
// chooses it, so that the two stay bit-identical.
template <int G>
__global__ void k_secular_noalloc_grp(const double* d, const double* w, const float* wf,
                                      const float* wl, const float* dh, const float* dl, int K,
                                      int* status, double* lam, double* gam, double* mu)
{
    const int tg = blockIdx.x * blockDim.x + threadIdx.x;
    if (((tg & ~31) / G) >= K) return;   // whole warps leave
    const int gl = threadIdx.x & (G - 1);
    const int i = tg / G;
    const bool act = i < K;
    double l = 0.0, g = 0.0, m = 0.0;
    int it, itdf;
    secular_root_group<G>(d, w, act ? K : 0, act ? i : 0, act, gl, &l, &g, &m, &it, &itdf, dh, dl,
                          wf, wl);
    if (act && gl == 0) {
        lam[i] = l;
        gam[i] = g;
        mu[i] = m;
        if (it > TD_SECULAR_MAXIT) atomicOr(status, TD_STATUS_NOTCONV);
    }
}

// Device memory of the current device (host, managed or another device's
// memory is rejected).
static bool noalloc_on_device(const void* p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

extern "C" int tdeig_secular_noalloc(int64_t K, const double* d, const double* z, double rho,
                                     double* lambda, double* gamma, double* mu, void* cuda_stream)
{
    if (K < 1 || K > TDEIG_NOALLOC_MAX_K) return TDEIG_EINVAL;
    if (!d || !z || !lambda || !gamma || !mu || !(rho > 0.0) || !isfinite(rho)) return TDEIG_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= TD_NOALLOC_MAX_DEVICES) {
        cudaGetLastError();
        return TDEIG_ECUDA;
    }
    if (!noalloc_on_device(d, dev) || !noalloc_on_device(z, dev) ||
        !noalloc_on_device(lambda, dev) || !noalloc_on_device(gamma, dev) ||
        !noalloc_on_device(mu, dev))
        return TDEIG_EINVAL;
    double* scratch;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, td_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return TDEIG_ECUDA;
            }
            g_noalloc_ptr[dev] = (double*)p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    double* w = scratch;
    float* f32 = (float*)(scratch + TD_NOALLOC_F32);
    float* wf = f32;
    float* wl = f32 + 3 * TDEIG_NOALLOC_MAX_K;
    float* dh = f32 + TDEIG_NOALLOC_MAX_K;
    float* dl = f32 + 2 * TDEIG_NOALLOC_MAX_K;
    int* status = (int*)(scratch + TD_NOALLOC_STATUS);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int k = (int)K;
    k_noalloc_weights<<<td_cdiv(k, 256), 256, 0, st>>>(d, z, rho, k, w, wf, wl, dh, dl, status);
    switch (secular_group(k, k)) {   // as tdeig_secular (a single merge of size K)
    case 4:
        k_secular_noalloc_grp<4><<<td_cdiv(k, 64), 256, 0, st>>>(d, w, wf, wl, dh, dl, k, status,
                                                                lambda, gamma, mu);
        break;
    case 8:
        k_secular_noalloc_grp<8><<<td_cdiv(k, 32), 256, 0, st>>>(d, w, wf, wl, dh, dl, k, status,
                                                                lambda, gamma, mu);
        break;
    case 16:
        k_secular_noalloc_grp<16><<<td_cdiv(k, 16), 256, 0, st>>>(d, w, wf, wl, dh, dl, k, status,
                                                                 lambda, gamma, mu);
        break;
    default:
        k_secular_noalloc<<<td_cdiv(k, 8), 256, 0, st>>>(d, w, wf, wl, dh, dl, k, status, lambda,
                                                          gamma, mu);
        break;
    }
    if (cudaGetLastError() != cudaSuccess) return TDEIG_ECUDA;
    int hs = 0;
    if (cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return TDEIG_ECUDA;
    return (hs & TD_STATUS_NOTCONV) ? TDEIG_ENOTCONV : TDEIG_OK;
}
