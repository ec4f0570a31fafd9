// Split-precision FP64 products on the tensor cores (see split.cuh for the
// scheme).  k_slice_exp finds the per-row exponent bounds of op(A) / per-column
// ones of op(B); k_slice writes the digits as BF16 or FP16 slices (K
// contiguous, padded to a multiple of 32); the products run in k_split_umma
// (kernels_umma.cu).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "split.cuh"

__device__ __forceinline__ double slice_load(const SliceDesc& d, int r, int k)
{
    if (k >= d.K1) return d.X2[r * d.sr2 + (long long)(k - d.K1) * d.sk2];
    if (d.mask && d.mask[r] == d.mask[k]) return 0.0;
    const long long c = d.gk ? d.gk[k] : k;
    return d.X[r * d.sr + c * d.sk];
}

// Grid: (operand, 32-row tile, k chunk of SE_K).  Each CTA takes the largest
// biased exponent field of its rows over its k chunk (integer maxima: FP64
// max/abs instructions would bind the kernel to the 1/64-rate FP64 pipe) and
// raises the rows' exponent bounds e (max |x| < 2^e, the field minus 1022) with
// atomicMax.  The bounds start at a large negative value; a row with no
// normal entry keeps it, which is harmless: every digit of that row is zero
// (subnormal entries are sliced as zero).  Eight independent loads per thread
// are in flight.
#define SE_K 1024

// Operand of flattened tile t: the last operand whose first tile is <= t
// (every launch covers exactly the tiles of its operands, whatever their sizes).
__device__ __forceinline__ int sl_operand(const SliceDesc* D, int nop, int t, bool exp_pass)
{
    int lo = 0, hi = nop - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((exp_pass ? D[mid].t_exp : D[mid].t_sl) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int exp_field(double x)
{
    return (__double2hiint(x) >> 20) & 0x7ff;
}

__global__ void k_slice_exp(const SliceDesc* D, int nop)
{
    const int t = blockIdx.x;
    const SliceDesc d = D[sl_operand(D, nop, t, true)];
    const int ry = (d.rows + 31) / 32;
    const int local = t - d.t_exp;
    const int r0 = (local % ry) * 32;
    const int kb = (local / ry) * SE_K;
    if (r0 >= d.rows || kb >= d.K) return;
    const int ke = min(d.K, kb + SE_K);
    __shared__ int red[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    if (d.sr == 1) {
        // rows contiguous: lane = row, warps stride over k
        const int r = r0 + tx;
        int mx = 0;
        if (r < d.rows)
            for (int k = kb + ty; k < ke; k += 64) {
                double v[8];
#pragma unroll
                for (int j = 0; j < 8; j++) v[j] = (k + 8 * j < ke) ? slice_load(d, r, k + 8 * j) : 0.0;
#pragma unroll
                for (int j = 0; j < 8; j++) mx = max(mx, exp_field(v[j]));
            }
        red[ty][tx] = mx;
        __syncthreads();
        if (ty == 0 && r < d.rows) {
            int m = 0;
            for (int w = 0; w < 8; w++) m = max(m, red[w][tx]);
            if (m > 0) atomicMax(d.e + r, m - 1022);
        }
    } else {
        // k contiguous: lane = k, warp ty handles rows ty, ty+8, ty+16, ty+24
        for (int q = 0; q < 4; q++) {
            const int r = r0 + ty + 8 * q;
            int m = 0;
            if (r < d.rows)
                for (int k = kb + tx; k < ke; k += 256) {
                    double v[8];
#pragma unroll
                    for (int j = 0; j < 8; j++) v[j] = (k + 32 * j < ke) ? slice_load(d, r, k + 32 * j) : 0.0;
#pragma unroll
                    for (int j = 0; j < 8; j++) m = max(m, exp_field(v[j]));
                }
            m = __reduce_max_sync(0xffffffffu, m);
            if (tx == 0 && r < d.rows && m > 0) atomicMax(d.e + r, m - 1022);
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

// Grid: (operand, 64-wide k tile, 64-row tile): the operand count (two per
// product, one product per merge) may exceed the 65535 limit of y and z.  The tile passes through shared
// memory (coalesced along whichever dimension of X is contiguous); then each
// thread turns 8 consecutive k of one row into digits and writes each slice's
// 8 values with one 16-byte store.  Shared rows hold 8 groups of 8 doubles,
// each group padded to 10 doubles, so a quarter-warp's 16-byte reads of the 8
// groups of a row fall in distinct banks (and the row stride of 82 doubles
// keeps the transposing stores at most 2-way).  Digits come from the 64-bit
// magnitude by 32-bit funnel shifts (beta s <= 56 < 64).
#define SL_T 64
#define SL_G 10   // padded group length (doubles)
#define SL_ROW (8 * SL_G + 2)   // +2: row stride 164 words

// The 64 x 64 tile of the operand at (r0, k0) into shared memory, rows of 8
// padded groups of 8 doubles; all 16 loads of a thread are issued before any
// shared-memory store.
__device__ __forceinline__ void slice_tile_load(const SliceDesc& d, double (*T)[SL_ROW], int r0, int k0)
{
    const int tid = threadIdx.x;
    double v[SL_T * SL_T / 256];
#pragma unroll
    for (int t = 0; t < SL_T * SL_T / 256; t++) {
        const int idx = tid + 256 * t;
        int r, k;
        if (d.sr == 1) { r = idx % SL_T; k = idx / SL_T; } else { k = idx % SL_T; r = idx / SL_T; }
        v[t] = (r0 + r < d.rows && k0 + k < d.K) ? slice_load(d, r0 + r, k0 + k) : 0.0;
    }
#pragma unroll
    for (int t = 0; t < SL_T * SL_T / 256; t++) {
        const int idx = tid + 256 * t;
        int r, k;
        if (d.sr == 1) { r = idx % SL_T; k = idx / SL_T; } else { k = idx % SL_T; r = idx / SL_T; }
        T[r][(k >> 3) * SL_G + (k & 7)] = v[t];
    }
}

// Grid: (operand, 64-wide k tile, 64-row tile): the operand count (two per
// product, one product per merge) may exceed the 65535 limit of y and z.  The
// tile passes through shared memory (coalesced along whichever dimension of X
// is contiguous); then each thread turns 8 consecutive k of one row into digits
// and writes each slice's 8 values with one 16-byte store.  Shared rows hold 8
// groups of 8 doubles, each group padded to 10 doubles, so a quarter-warp's
// 16-byte reads of the 8 groups of a row fall in distinct banks (and the row
// stride of 82 doubles keeps the transposing stores at most 2-way).  Digits
// come from the 64-bit magnitude by 32-bit funnel shifts (beta s <= 56 < 64).
// General form (any beta, BF16 or FP16 slices).
__global__ void __launch_bounds__(256) k_slice(const SliceDesc* D, int nop)
{
    const int t = blockIdx.x;   // flattened (operand, 64-row tile, 64-wide k tile)
    const SliceDesc d = D[sl_operand(D, nop, t, false)];
    const int ky = (d.Kp + SL_T - 1) / SL_T;
    const int k0 = ((t - d.t_sl) % ky) * SL_T, r0 = ((t - d.t_sl) / ky) * SL_T;
    if (k0 >= d.Kp || r0 >= d.rows) return;
    __shared__ __align__(16) double T[SL_T][SL_ROW];
    const int tid = threadIdx.x;
    slice_tile_load(d, T, r0, k0);
    __syncthreads();
    const int bs = d.beta * d.s;
    const unsigned mask = (1u << d.beta) - 1u;
#pragma unroll
    for (int i = 0; i < (SL_T * SL_T / 8) / 256; i++) {
        const int u = tid + 256 * i;
        const int r = u / (SL_T / 8), kg = u % (SL_T / 8);
        const int row = r0 + r, kk = k0 + kg * 8;
        if (row >= d.rows || kk >= d.Kp) continue;
        const int e = d.e[row];
        unsigned mlo[8], mhi[8];
        float sg[8];
        const double2* src = (const double2*)&T[r][kg * SL_G];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const double2 x2 = src[j];
            const long long m0 = slice_mag(x2.x, e, bs), m1 = slice_mag(x2.y, e, bs);
            mlo[2 * j] = (unsigned)m0; mhi[2 * j] = (unsigned)(m0 >> 32);
            mlo[2 * j + 1] = (unsigned)m1; mhi[2 * j + 1] = (unsigned)(m1 >> 32);
            // signs from the bit patterns (an FP64 compare issues on the slow FP64 pipe)
            sg[2 * j] = (__double2hiint(x2.x) < 0) ? -1.0f : 1.0f;
            sg[2 * j + 1] = (__double2hiint(x2.y) < 0) ? -1.0f : 1.0f;
        }
        for (int p = 0; p < d.s; p++) {
            const float sc = __int_as_float((127 - d.beta * p) << 23);   // 2^(-beta p), exact
            const int sh = d.beta * (d.s - 1 - p);
            unsigned short h[8];
#pragma unroll
            for (int j = 0; j < 8; j++) {
                // bits [sh, sh + beta) of the 64-bit magnitude
                const unsigned w = sh >= 32 ? (mhi[j] >> (sh - 32)) : __funnelshift_r(mlo[j], mhi[j], sh);
                // the digit as a float without a conversion instruction: 2^23 + t - 2^23
                const float t = __uint_as_float(0x4B000000u | (w & mask)) - 8388608.0f;
                // t_p 2^(-beta p): exact in the slice type (beta <= 8 BF16, <= 11 FP16)
                const float val = t * (sg[j] * sc);
                // at most 8 significant bits: the BF16 pattern is the top half of the FP32 one
                h[j] = d.f16 ? __half_as_ushort(__float2half_rn(val))
                             : (unsigned short)(__float_as_uint(val) >> 16);
            }
            uint4 w4;
            w4.x = (unsigned)h[0] | ((unsigned)h[1] << 16);
            w4.y = (unsigned)h[2] | ((unsigned)h[3] << 16);
            w4.z = (unsigned)h[4] | ((unsigned)h[5] << 16);
            w4.w = (unsigned)h[6] | ((unsigned)h[7] << 16);
            *(uint4*)(d.S + ((size_t)p * d.rows + row) * d.Kp + kk) = w4;
        }
    }
}

// The 7-bit-digit BF16 form with the slice count fixed at compile time, in
// balanced digits.  The magnitude m = floor(|x| 2^(7S - e)) is written as
//   m = t_0 128^(S-1) + sum_{p>=1} t_p 128^(S-1-p),  t_p in [-64, 63] (p >= 1),
//   t_0 in [0, 128],
// read off m + B, B = 64 sum_{j<S-1} 128^j: digit p >= 1 is u_p - 64 with u_p
// the base-128 digit of m + B, and t_0 its top part.  Smaller digits bound a
// level's integer sum per k by 2 * 128 * 64 + 6 * 64^2 = 40960 (at most 8 pairs,
// two of them with t_0), so it stays exact in FP32 over 384 k (the unbalanced
// digits 0..127 allowed 128 k).  Two digits of neighbouring entries are packed
// as the BF16 pair (128 + u0, 128 + u1) (bit patterns 0x4300 | u) and turned
// into (u0 - 64, u1 - 64) 2^(-7p) by one fma.rn.bf16x2 with the exact constants
// 2^(-7p) and -192 2^(-7p); t_0 <= 128 has at most 8 significant bits and is
// converted exactly through FP32.  The entries' signs are then set by an XOR of
// the sign bits.  Every value is exact.
template <int S>
__global__ void __launch_bounds__(256, 4) k_slice7(const SliceDesc* D, int nop)
{
    const int t = blockIdx.x;   // flattened (operand, 64-row tile, 64-wide k tile)
    const SliceDesc d = D[sl_operand(D, nop, t, false)];
    const int ky = (d.Kp + SL_T - 1) / SL_T;
    const int k0 = ((t - d.t_sl) % ky) * SL_T, r0 = ((t - d.t_sl) / ky) * SL_T;
    if (k0 >= d.Kp || r0 >= d.rows) return;
    __shared__ __align__(16) double T[SL_T][SL_ROW];
    const int tid = threadIdx.x;
    slice_tile_load(d, T, r0, k0);
    __syncthreads();
    constexpr int BS = 7 * S;
    // 64 in every base-128 digit below the top one
    unsigned long long B = 0;
#pragma unroll
    for (int j = 0; j < S - 1; j++) B |= 64ull << (7 * j);
#pragma unroll
    for (int i = 0; i < (SL_T * SL_T / 8) / 256; i++) {
        const int u = tid + 256 * i;
        const int r = u / (SL_T / 8), kg = u % (SL_T / 8);
        const int row = r0 + r, kk = k0 + kg * 8;
        if (row >= d.rows || kk >= d.Kp) continue;
        const int e = d.e[row];
        unsigned long long m[8];
        unsigned sgn[4];   // sign bits of the pairs at bits 15 and 31
        const double2* src = (const double2*)&T[r][kg * SL_G];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const double2 x2 = src[j];
            m[2 * j] = (unsigned long long)slice_mag(x2.x, e, BS) + B;
            m[2 * j + 1] = (unsigned long long)slice_mag(x2.y, e, BS) + B;
            sgn[j] = (((unsigned)__double2hiint(x2.x) >> 31) << 15) | ((unsigned)__double2hiint(x2.y) & 0x80000000u);
        }
        {
            // top digit t_0 = (m + B) >> 7 (S - 1) in [0, 128], exact through FP32
            unsigned w[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const unsigned t0 = (unsigned)(m[2 * j] >> (7 * (S - 1)));
                const unsigned t1 = (unsigned)(m[2 * j + 1] >> (7 * (S - 1)));
                const unsigned h0 = __float_as_uint(__uint_as_float(0x4B000000u | t0) - 8388608.0f) >> 16;
                const unsigned h1 = __float_as_uint(__uint_as_float(0x4B000000u | t1) - 8388608.0f) >> 16;
                w[j] = (h0 | (h1 << 16)) ^ sgn[j];
            }
            *(uint4*)(d.S + (size_t)row * d.Kp + kk) = make_uint4(w[0], w[1], w[2], w[3]);
        }
#pragma unroll
        for (int p = 1; p < S; p++) {
            const int sh = 7 * (S - 1 - p);
            const unsigned sc = (unsigned)(127 - 7 * p) << 7;                     // BF16 2^(-7p)
            const unsigned nc = ((unsigned)(134 - 7 * p) << 7) | 0x8040u;         // BF16 -192 2^(-7p)
            const __nv_bfloat162 sc2 = __halves2bfloat162(__ushort_as_bfloat16((unsigned short)sc),
                                                          __ushort_as_bfloat16((unsigned short)sc));
            const __nv_bfloat162 nc2 = __halves2bfloat162(__ushort_as_bfloat16((unsigned short)nc),
                                                          __ushort_as_bfloat16((unsigned short)nc));
            unsigned w[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const unsigned d0 = (unsigned)(m[2 * j] >> sh) & 127u;
                const unsigned d1 = (unsigned)(m[2 * j + 1] >> sh) & 127u;
                const unsigned pk = d0 | (d1 << 16) | 0x43004300u;
                __nv_bfloat162 x = *reinterpret_cast<const __nv_bfloat162*>(&pk);
                x = __hfma2(x, sc2, nc2);
                w[j] = *reinterpret_cast<const unsigned*>(&x) ^ sgn[j];
            }
            *(uint4*)(d.S + ((size_t)p * d.rows + row) * d.Kp + kk) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
void split_free(SplitWS& w)
{
    if (w.base) cudaFree(w.base);
    w.base = nullptr;
    w.cap = 0;
}

static size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
static PFN_cuTensorMapEncodeTiled_v12000 tmap_encoder()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        else
            cudaGetLastError();
    }
    return fn;
}

// 3-D map over the s slices of an operand: (k: Kp, row: rows, slice: s), 16-bit
// elements, box (UM_BK, box_rows, s), 64-byte swizzle, zero fill past the ends.
static bool encode_slices(CUtensorMap* m, const void* base, int Kp, int rows, int s, int box_rows)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = tmap_encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)s};
    const cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)rows * Kp * 2};
    const cuuint32_t box[3] = {UM_BK, (cuuint32_t)box_rows, (cuuint32_t)s};
    const cuuint32_t es[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 3, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

SplitPrec split_prec(int kind, int bits)
{
    SplitPrec p;
    switch (kind) {
    case SPLIT_BF16X2:   // two 8-bit digits: levels 0 and 1, 2 x 255^2 x 128 < 2^24
        p.beta = 8; p.s = 2; p.chunk = 128; p.f16 = 0; p.nacc = 2;
        break;
    case SPLIT_FP16X2:   // two 11-bit digits: FP32 accumulation rounds
        p.beta = 11; p.s = 2; p.chunk = UM_BK; p.f16 = 1; p.nacc = 2;
        break;
    default:             // balanced 7-bit digits, s <= 8: every level exact over 384 k,
                         // (2 x 128 x 64 + 6 x 64^2) x 384 < 2^24
        p.beta = 7; p.s = (bits + 6) / 7; p.chunk = 384; p.f16 = 0; p.nacc = p.s;
        break;
    }
    return p;
}

double split_launch_gemm(const std::vector<GemmDesc>& gin, SplitWS& ws, cudaStream_t st, int* rc,
                         int* status, int kind, int bits)
{
    const SplitPrec pr = split_prec(kind, bits);
    *rc = TDEIG_OK;
    std::vector<GemmDesc> g;
    for (const GemmDesc& d : gin)
        if (d.M > 0 && d.N > 0) g.push_back(d);
    if (g.empty()) return 0.0;
    // scratch: slices and exponents of both operands of every problem, descriptors
    size_t bytes = al256(g.size() * 2 * sizeof(SliceDesc)) + al256(g.size() * sizeof(SplitGemmDesc)) +
                   al256(g.size() * sizeof(int)) + al256(g.size() * 2 * sizeof(CUtensorMap));
    std::vector<int> betas(g.size()), ss(g.size()), kps(g.size());
    double flops = 0.0, tflops = 0.0, sbytes = 0.0, ebytes = 0.0;
    for (size_t i = 0; i < g.size(); i++) {
        betas[i] = pr.beta;
        ss[i] = pr.s;
        const int Kt = g[i].Kd + g[i].Kd2;
        kps[i] = std::max(32, ((Kt + 31) / 32) * 32);
        bytes += al256((size_t)ss[i] * g[i].M * kps[i] * 2) + al256((size_t)ss[i] * g[i].N * kps[i] * 2);
        bytes += ((size_t)g[i].M + g[i].N) * 4;
        flops += 2.0 * g[i].M * g[i].N * Kt;
        tflops += 2.0 * g[i].M * g[i].N * Kt * (ss[i] * (ss[i] + 1) / 2);
        // algorithmic traffic: every operand element read once by each slicing kernel,
        // 2 s bytes of slices written per padded element
        const double elems = (double)(g[i].M + g[i].N) * Kt;
        sbytes += 8.0 * elems + 2.0 * ss[i] * (double)(g[i].M + g[i].N) * kps[i];
        ebytes += 8.0 * elems;
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
    // exponents of every operand row in one region, filled with 0xC0 bytes
    // (-1061109568: far below any exponent, and two of them still add without
    // overflow) before k_slice_exp raises them
    size_t erows = 0;
    for (size_t i = 0; i < g.size(); i++) erows += (size_t)g[i].M + g[i].N;
    int* ebase = (int*)take(erows * 4);
    size_t eoff = 0;
    SliceDesc* dsl = (SliceDesc*)take(g.size() * 2 * sizeof(SliceDesc));
    SplitGemmDesc* dsg = (SplitGemmDesc*)take(g.size() * sizeof(SplitGemmDesc));
    int* dt0 = (int*)take(g.size() * sizeof(int));
    CUtensorMap* dtm = (CUtensorMap*)take(g.size() * 2 * sizeof(CUtensorMap));   // 256-aligned
    std::vector<CUtensorMap> tm(g.size() * 2);
    std::vector<SliceDesc> sl;
    std::vector<SplitGemmDesc> sg;
    int maxrows = 0, maxkp = 0, tiles = 0;
    for (size_t i = 0; i < g.size(); i++) {
        const GemmDesc& d = g[i];
        SliceDesc a;
        memset(&a, 0, sizeof(a));
        a.X = d.A;
        a.mask = d.amask;
        if (!d.transA) { a.sr = 1; a.sk = d.lda; a.gk = d.acol; }
        else { a.sr = d.lda; a.sk = 1; a.gk = nullptr; }
        a.K1 = d.Kd;
        if (d.Kd2 > 0) {
            a.X2 = d.A2;
            if (!d.transA2) { a.sr2 = 1; a.sk2 = d.lda2; } else { a.sr2 = d.lda2; a.sk2 = 1; }
        }
        a.rows = d.M; a.K = d.Kd + d.Kd2; a.Kp = kps[i]; a.s = ss[i]; a.beta = betas[i]; a.f16 = pr.f16;
        a.S = (__nv_bfloat16*)take((size_t)ss[i] * d.M * kps[i] * 2);
        a.e = ebase + eoff;
        eoff += d.M;
        SliceDesc b;
        memset(&b, 0, sizeof(b));
        b.X = d.B;
        if (!d.transB) { b.sr = d.ldb; b.sk = 1; } else { b.sr = 1; b.sk = d.ldb; }
        b.K1 = d.Kd;
        if (d.Kd2 > 0) {
            b.X2 = d.B2;
            if (!d.transB2) { b.sr2 = d.ldb2; b.sk2 = 1; } else { b.sr2 = 1; b.sk2 = d.ldb2; }
        }
        b.rows = d.N; b.K = d.Kd + d.Kd2; b.Kp = kps[i]; b.s = ss[i]; b.beta = betas[i]; b.f16 = pr.f16;
        b.S = (__nv_bfloat16*)take((size_t)ss[i] * d.N * kps[i] * 2);
        b.e = ebase + eoff;
        eoff += d.N;
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
        s.chunk = pr.chunk; s.f16 = pr.f16;
        if (!encode_slices(&tm[2 * i], a.S, kps[i], d.M, ss[i], UM_BM) ||
            !encode_slices(&tm[2 * i + 1], b.S, kps[i], d.N, ss[i], UM_BN)) {
            *rc = TDEIG_ECUDA;
            return 0.0;
        }
        s.tmA = dtm + 2 * i;
        s.tmB = dtm + 2 * i + 1;
        s.tiles_m = td_cdiv(d.M, UM_BM);
        s.tile0 = tiles;
        tiles += s.tiles_m * td_cdiv(d.N, UM_BN);
        sg.push_back(s);
    }
    // flattened tile lists of the two slicing launches
    long long nexp = 0, nsl = 0;
    for (auto& o : sl) {
        o.t_exp = (int)nexp;
        o.t_sl = (int)nsl;
        nexp += (long long)td_cdiv(o.rows, 32) * td_cdiv(o.K, SE_K);
        nsl += (long long)td_cdiv(o.Kp, SL_T) * td_cdiv(o.rows, SL_T);
    }
    if (nexp >= (1ll << 31) || nsl >= (1ll << 31)) {
        *rc = TDEIG_EINVAL;
        return 0.0;
    }
    std::vector<int> t0(sg.size());
    for (size_t i = 0; i < sg.size(); i++) t0[i] = sg[i].tile0;
    if (cudaMemcpyAsync(dtm, tm.data(), tm.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(dt0, t0.data(), t0.size() * sizeof(int), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(dsl, sl.data(), sl.size() * sizeof(SliceDesc), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(dsg, sg.data(), sg.size() * sizeof(SplitGemmDesc), cudaMemcpyHostToDevice, st) !=
            cudaSuccess) {
        *rc = TDEIG_ECUDA;
        return 0.0;
    }
    if (cudaMemsetAsync(ebase, 0xC0, erows * 4, st) != cudaSuccess) {
        *rc = TDEIG_ECUDA;
        return 0.0;
    }
    const int nop = (int)sl.size();
    td_prof_begin(st);
    k_slice_exp<<<(unsigned)nexp, 256, 0, st>>>(dsl, nop);
    td_prof_end(st, "k_slice_exp");
    const unsigned gs = (unsigned)nsl;
    td_prof_begin(st);
    if (pr.beta == 7 && !pr.f16) {
        switch (pr.s) {
        case 1: k_slice7<1><<<gs, 256, 0, st>>>(dsl, nop); break;
        case 2: k_slice7<2><<<gs, 256, 0, st>>>(dsl, nop); break;
        case 3: k_slice7<3><<<gs, 256, 0, st>>>(dsl, nop); break;
        case 4: k_slice7<4><<<gs, 256, 0, st>>>(dsl, nop); break;
        case 5: k_slice7<5><<<gs, 256, 0, st>>>(dsl, nop); break;
        case 6: k_slice7<6><<<gs, 256, 0, st>>>(dsl, nop); break;
        case 7: k_slice7<7><<<gs, 256, 0, st>>>(dsl, nop); break;
        default: k_slice7<8><<<gs, 256, 0, st>>>(dsl, nop); break;
        }
    } else {
        k_slice<<<gs, 256, 0, st>>>(dsl, nop);
    }
    td_prof_end(st, "k_slice");
    umma_launch(dsg, dt0, (int)sg.size(), tiles, pr.s, pr.nacc, status, st);
    TdCtx& cx = td_ctx();
    if (cx.prof.on) {
        // [tiles, k-blocks over all tiles, slices, problems, tensor flops]
        double kbl = 0.0;
        for (size_t i = 0; i < g.size(); i++)
            kbl += (double)sg[i].tiles_m * td_cdiv(g[i].N, UM_BN) * (kps[i] / UM_BK);
        char nb[160];
        snprintf(nb, sizeof(nb), "[%d,%.0f,%d,%d,%.6e]", tiles, kbl, pr.s, (int)g.size(), tflops);
        td_prof_note(nb);
    }
    cx.split_tensor_flops += tflops;
    cx.split_slice_bytes += sbytes;
    cx.split_exp_bytes += ebytes;
    if (cudaGetLastError() != cudaSuccess) *rc = TDEIG_ECUDA;
    return flops;
}
