// Split-precision FP64 products on the tensor cores (see split.cuh for the
// scheme).  k_slice_exp finds the per-row exponent bounds of op(A) / per-column
// ones of op(B); k_slice writes the integer BF16 digits (K contiguous, padded
// to a multiple of 32); k_split_gemm runs, for every output tile, the slice-pair
// products with p + q <= s - 1 on mma.sync m16n8k16 (BF16 in, FP32 exact
// accumulation), accumulates them in a double-float sum and writes FP64.
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "split.cuh"

void split_params(int K, int* beta, int* s)
{
    int b = 8;
    while (b > 1 && (double)((1 << b) - 1) * (double)((1 << b) - 1) * (double)std::max(K, 1) > 16777216.0)
        b--;
    *beta = b;
    *s = (TD_SPLIT_BITS + b - 1) / b;
}

// element (r, k) of the operand being sliced: X[r*sr + col(k)*sk], col(k) = gk ? gk[k] : k
struct SliceDesc {
    const double* X;
    const int* gk;
    long long sr, sk;
    int rows, K, Kp, s, beta;
    __nv_bfloat16* S;   // slice p, row r at S + (p * rows + r) * Kp
    int* e;             // exponent bound per row: max |row| < 2^e
};

__device__ __forceinline__ double slice_load(const SliceDesc& d, int r, int k)
{
    const long long c = d.gk ? d.gk[k] : k;
    return d.X[r * d.sr + c * d.sk];
}

__global__ void k_slice_exp(const SliceDesc* D)
{
    const SliceDesc d = D[blockIdx.y];
    const int r0 = blockIdx.x * 32;
    if (r0 >= d.rows) return;
    __shared__ double red[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    double mx[4] = {0.0, 0.0, 0.0, 0.0};
    if (d.sr == 1) {
        // rows contiguous: lane = row, warps stride over k
        const int r = r0 + tx;
        if (r < d.rows)
            for (int k = ty; k < d.K; k += 8) mx[0] = fmax(mx[0], fabs(slice_load(d, r, k)));
        red[ty][tx] = mx[0];
        __syncthreads();
        if (ty == 0 && r < d.rows) {
            double m = 0.0;
            for (int w = 0; w < 8; w++) m = fmax(m, red[w][tx]);
            int ex = 0;
            if (m > 0.0) frexp(m, &ex);
            d.e[r] = ex;
        }
    } else {
        // k contiguous: lane = k, warp ty handles rows ty, ty+8, ty+16, ty+24
        for (int q = 0; q < 4; q++) {
            const int r = r0 + ty + 8 * q;
            double m = 0.0;
            if (r < d.rows)
                for (int k = tx; k < d.K; k += 32) m = fmax(m, fabs(slice_load(d, r, k)));
            m = td_warp_max(m);
            if (tx == 0 && r < d.rows) {
                int ex = 0;
                if (m > 0.0) frexp(m, &ex);
                d.e[r] = ex;
            }
        }
    }
}

// floor(|x| 2^(beta s - e)) as an integer; |x| < 2^e, beta s <= 52
__device__ __forceinline__ long long slice_mag(double x, int e, int bs)
{
    const long long b = __double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff);
    if (ex == 0) return 0;
    const long long mant = (b & 0xFFFFFFFFFFFFFLL) | (1LL << 52);
    const int sh = ex - 1075 + bs - e;
    if (sh >= 0) return mant << min(sh, 10);
    if (sh <= -63) return 0;
    return mant >> (-sh);
}

__global__ void k_slice(const SliceDesc* D)
{
    const SliceDesc d = D[blockIdx.z];
    const int k0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    if (k0 >= d.Kp || r0 >= d.rows) return;
    __shared__ double T[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int q = ty; q < 32; q += 8) {
        // T[row][k]; coalesced along the contiguous dimension of X
        int r, k;
        if (d.sr == 1) { r = r0 + tx; k = k0 + q; } else { r = r0 + q; k = k0 + tx; }
        double v = 0.0;
        if (r < d.rows && k < d.K) v = slice_load(d, r, k);
        if (d.sr == 1) T[tx][q] = v; else T[q][tx] = v;
    }
    __syncthreads();
    const int bs = d.beta * d.s;
    const long long mask = (1LL << d.beta) - 1;
    for (int q = ty; q < 32; q += 8) {
        const int r = r0 + q, k = k0 + tx;
        if (r >= d.rows) continue;
        const double x = T[q][tx];
        const long long M = slice_mag(x, d.e[r], bs);
        const float sg = (x < 0.0) ? -1.0f : 1.0f;
        for (int p = 0; p < d.s; p++) {
            const long long dig = (M >> (d.beta * (d.s - 1 - p))) & mask;
            d.S[((size_t)p * d.rows + r) * d.Kp + k] = __float2bfloat16_rn(sg * (float)dig);
        }
    }
}

// ---------------------------------------------------------------------------
// Grouped slice-pair product.  Tile 128 x 64, BK 32, 8 warps (4 x 2), warp tile
// 32 x 32 = 2 x 4 mma.m16n8k16 tiles; 3-stage cp.async pipeline; shared rows
// padded to 80 bytes so ldmatrix reads are conflict-free.
// ---------------------------------------------------------------------------
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
    int rsplit, ktop_end, kbot_beg;
    int tile0, tiles_m;
};

#define SG_BM 128
#define SG_BN 64
#define SG_BK 32
#define SG_LD 40   // padded row length in bf16 elements (80 bytes)
#define SG_ST 3

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, bool valid)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n));
}

__device__ __forceinline__ void ldsm_x4(unsigned& r0, unsigned& r1, unsigned& r2, unsigned& r3,
                                        const void* p)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(s));
}

__device__ __forceinline__ void mma_bf16(float* c, const unsigned* a, unsigned b0, unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(256) k_split_gemm(const SplitGemmDesc* G, int ng)
{
    __shared__ __align__(128) __nv_bfloat16 sA[SG_ST][SG_BM][SG_LD];
    __shared__ __align__(128) __nv_bfloat16 sB[SG_ST][SG_BN][SG_LD];
    const int bid = blockIdx.x;
    int lo = 0, hi = ng - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (G[mid].tile0 <= bid) lo = mid; else hi = mid - 1;
    }
    const SplitGemmDesc g = G[lo];
    const int local = bid - g.tile0;
    const int tm = local % g.tiles_m, tn = local / g.tiles_m;
    const int row0 = tm * SG_BM, col0 = tn * SG_BN;
    if (row0 >= g.M || col0 >= g.N) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp & 3) * 32, wn = (warp >> 2) * 32;
    int kb0 = 0, kb1 = g.Kp;
    if (g.rsplit > 0) {
        if (row0 >= g.rsplit) kb0 = (g.kbot_beg / SG_BK) * SG_BK;
        if (row0 + SG_BM <= g.rsplit) kb1 = min(g.Kp, ((g.ktop_end + SG_BK - 1) / SG_BK) * SG_BK);
    }
    float hi_acc[2][4][4], lo_acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 4; b++)
#pragma unroll
            for (int c = 0; c < 4; c++) { hi_acc[a][b][c] = 0.f; lo_acc[a][b][c] = 0.f; }

    for (int p = 0; p < g.s; p++) {
        for (int q = 0; p + q < g.s; q++) {
            const __nv_bfloat16* Ap = g.SA + (size_t)p * g.M * g.Kp;
            const __nv_bfloat16* Bq = g.SB + (size_t)q * g.N * g.Kp;
            float acc[2][4][4];
#pragma unroll
            for (int a = 0; a < 2; a++)
#pragma unroll
                for (int b = 0; b < 4; b++)
#pragma unroll
                    for (int c = 0; c < 4; c++) acc[a][b][c] = 0.f;
            auto load = [&](int st, int k0) {
#pragma unroll
                for (int i = 0; i < 2; i++) {
                    const int ch = tid + 256 * i;          // 512 chunks of A: 128 rows x 4
                    const int r = ch >> 2, c = ch & 3;
                    const int gr = row0 + r;
                    const bool v = gr < g.M;
                    cp_async16(&sA[st][r][c * 8], Ap + (size_t)(v ? gr : 0) * g.Kp + k0 + c * 8, v);
                }
                {
                    const int r = tid >> 2, c = tid & 3;  // 256 chunks of B: 64 rows x 4
                    const int gc = col0 + r;
                    const bool v = gc < g.N;
                    cp_async16(&sB[st][r][c * 8], Bq + (size_t)(v ? gc : 0) * g.Kp + k0 + c * 8, v);
                }
                asm volatile("cp.async.commit_group;\n" ::);
            };
            const int nkb = (kb1 - kb0) / SG_BK;
            __syncthreads();   // the previous pair's last stage reads are done
            for (int i = 0; i < SG_ST - 1; i++) {
                if (i < nkb) load(i, kb0 + i * SG_BK);
                else asm volatile("cp.async.commit_group;\n" ::);
            }
            for (int it = 0; it < nkb; it++) {
                asm volatile("cp.async.wait_group %0;\n" ::"n"(SG_ST - 2));
                __syncthreads();
                const int nxt = it + SG_ST - 1;
                if (nxt < nkb) load(nxt % SG_ST, kb0 + nxt * SG_BK);
                else asm volatile("cp.async.commit_group;\n" ::);
                const int st = it % SG_ST;
#pragma unroll
                for (int kk = 0; kk < SG_BK; kk += 16) {
                    unsigned af[2][4], bf[4][2];
#pragma unroll
                    for (int mi = 0; mi < 2; mi++) {
                        const int r = wm + mi * 16 + (lane & 15);
                        const int c = kk + (lane >> 4) * 8;
                        ldsm_x4(af[mi][0], af[mi][1], af[mi][2], af[mi][3], &sA[st][r][c]);
                    }
#pragma unroll
                    for (int nj = 0; nj < 2; nj++) {
                        const int r = wn + nj * 16 + (lane & 7) + ((lane >> 4) << 3);
                        const int c = kk + ((lane >> 3) & 1) * 8;
                        unsigned r0, r1, r2, r3;
                        ldsm_x4(r0, r1, r2, r3, &sB[st][r][c]);
                        bf[nj * 2][0] = r0; bf[nj * 2][1] = r1;
                        bf[nj * 2 + 1][0] = r2; bf[nj * 2 + 1][1] = r3;
                    }
#pragma unroll
                    for (int mi = 0; mi < 2; mi++)
#pragma unroll
                        for (int ni = 0; ni < 4; ni++) mma_bf16(acc[mi][ni], af[mi], bf[ni][0], bf[ni][1]);
                }
            }
            // exact slice-pair sums -> double-float accumulation
            const float sc = ldexpf(1.0f, -g.beta * (p + q + 2));
#pragma unroll
            for (int a = 0; a < 2; a++)
#pragma unroll
                for (int b = 0; b < 4; b++)
#pragma unroll
                    for (int c = 0; c < 4; c++) {
                        const float x = acc[a][b][c] * sc;
                        const float h = hi_acc[a][b][c];
                        const float s2 = h + x;
                        const float bb = s2 - h;
                        const float err = (h - (s2 - bb)) + (x - bb);
                        hi_acc[a][b][c] = s2;
                        lo_acc[a][b][c] += err;
                    }
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
    // write: C[row, ccol(col)] = alpha 2^(ea+eb) (hi + lo) + betac C
    const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int b = 0; b < 4; b++)
#pragma unroll
            for (int c = 0; c < 4; c++) {
                const int row = row0 + wm + a * 16 + gq + ((c >> 1) << 3);
                const int col = col0 + wn + b * 8 + tq * 2 + (c & 1);
                if (row >= g.M || col >= g.N) continue;
                const double v = ldexp((double)hi_acc[a][b][c] + (double)lo_acc[a][b][c],
                                       g.ea[row] + g.eb[col]);
                double* out = g.C + (size_t)(g.ccol ? g.ccol[col] : col) * g.ldc + row;
                *out = g.betac != 0.0 ? g.alpha * v + g.betac * (*out) : g.alpha * v;
            }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
double g_split_tensor_flops = 0.0;

void split_free(SplitWS& w)
{
    if (w.base) cudaFree(w.base);
    w.base = nullptr;
    w.cap = 0;
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

double split_launch_gemm(const std::vector<GemmDesc>& gin, SplitWS& ws, cudaStream_t st, int* rc)
{
    *rc = TDEIG_OK;
    std::vector<GemmDesc> g;
    for (const GemmDesc& d : gin)
        if (d.M > 0 && d.N > 0) g.push_back(d);
    if (g.empty()) return 0.0;
    // scratch: slices and exponents of both operands of every problem, descriptors
    size_t bytes = al256(g.size() * 2 * sizeof(SliceDesc)) + al256(g.size() * sizeof(SplitGemmDesc));
    std::vector<int> betas(g.size()), ss(g.size()), kps(g.size());
    double flops = 0.0, tflops = 0.0;
    for (size_t i = 0; i < g.size(); i++) {
        split_params(std::max(g[i].Kd, 1), &betas[i], &ss[i]);
        kps[i] = std::max(SG_BK, ((g[i].Kd + SG_BK - 1) / SG_BK) * SG_BK);
        bytes += al256((size_t)ss[i] * g[i].M * kps[i] * 2) + al256((size_t)ss[i] * g[i].N * kps[i] * 2);
        bytes += al256((size_t)g[i].M * 4) + al256((size_t)g[i].N * 4);
        flops += 2.0 * g[i].M * g[i].N * g[i].Kd;
        tflops += 2.0 * g[i].M * g[i].N * g[i].Kd * (ss[i] * (ss[i] + 1) / 2);
    }
    if (bytes > ws.cap) {
        cudaStreamSynchronize(st);
        split_free(ws);
        const size_t want = bytes + bytes / 4;
        if (cudaMalloc(&ws.base, want) != cudaSuccess) {
            cudaGetLastError();
            *rc = TDEIG_ENOMEM;
            return 0.0;
        }
        ws.cap = want;
    }
    char* p = ws.base;
    auto take = [&](size_t n) { char* r = p; p += al256(n); return r; };
    SliceDesc* dsl = (SliceDesc*)take(g.size() * 2 * sizeof(SliceDesc));
    SplitGemmDesc* dsg = (SplitGemmDesc*)take(g.size() * sizeof(SplitGemmDesc));
    std::vector<SliceDesc> sl;
    std::vector<SplitGemmDesc> sg;
    int maxrows = 0, maxkp = 0, tiles = 0;
    for (size_t i = 0; i < g.size(); i++) {
        const GemmDesc& d = g[i];
        SliceDesc a;
        memset(&a, 0, sizeof(a));
        a.X = d.A;
        if (!d.transA) { a.sr = 1; a.sk = d.lda; a.gk = d.acol; }
        else { a.sr = d.lda; a.sk = 1; a.gk = nullptr; }
        a.rows = d.M; a.K = d.Kd; a.Kp = kps[i]; a.s = ss[i]; a.beta = betas[i];
        a.S = (__nv_bfloat16*)take((size_t)ss[i] * d.M * kps[i] * 2);
        a.e = (int*)take((size_t)d.M * 4);
        SliceDesc b;
        memset(&b, 0, sizeof(b));
        b.X = d.B;
        if (!d.transB) { b.sr = d.ldb; b.sk = 1; } else { b.sr = 1; b.sk = d.ldb; }
        b.rows = d.N; b.K = d.Kd; b.Kp = kps[i]; b.s = ss[i]; b.beta = betas[i];
        b.S = (__nv_bfloat16*)take((size_t)ss[i] * d.N * kps[i] * 2);
        b.e = (int*)take((size_t)d.N * 4);
        sl.push_back(a);
        sl.push_back(b);
        maxrows = std::max(maxrows, std::max(d.M, d.N));
        maxkp = std::max(maxkp, kps[i]);
        SplitGemmDesc s;
        memset(&s, 0, sizeof(s));
        s.SA = a.S; s.SB = b.S; s.ea = a.e; s.eb = b.e;
        s.M = d.M; s.N = d.N; s.Kp = kps[i]; s.s = ss[i]; s.beta = betas[i];
        s.C = d.C; s.ldc = d.ldc; s.ccol = d.ccol; s.alpha = d.alpha; s.betac = d.beta;
        s.rsplit = d.rsplit; s.ktop_end = d.ktop_end; s.kbot_beg = d.kbot_beg;
        s.tiles_m = td_cdiv(d.M, SG_BM);
        s.tile0 = tiles;
        tiles += s.tiles_m * td_cdiv(d.N, SG_BN);
        sg.push_back(s);
    }
    if (cudaMemcpyAsync(dsl, sl.data(), sl.size() * sizeof(SliceDesc), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(dsg, sg.data(), sg.size() * sizeof(SplitGemmDesc), cudaMemcpyHostToDevice, st) !=
            cudaSuccess) {
        *rc = TDEIG_ECUDA;
        return 0.0;
    }
    const unsigned ry = (unsigned)td_cdiv(maxrows, 32);
    td_prof_begin(st);
    k_slice_exp<<<dim3(ry, (unsigned)sl.size()), 256, 0, st>>>(dsl);
    td_prof_end(st, "k_slice_exp");
    td_prof_begin(st);
    k_slice<<<dim3((unsigned)(maxkp / 32), ry, (unsigned)sl.size()), 256, 0, st>>>(dsl);
    td_prof_end(st, "k_slice");
    td_prof_begin(st);
    k_split_gemm<<<tiles, 256, 0, st>>>(dsg, (int)sg.size());
    td_prof_end(st, "k_split_gemm");
    g_split_tensor_flops += tflops;
    if (cudaGetLastError() != cudaSuccess) *rc = TDEIG_ECUDA;
    return flops;
}
