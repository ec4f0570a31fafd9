// Split-precision FP64 products on the tensor cores (see split.cuh for the
// scheme).  k_slice_exp finds the per-row exponent bounds of op(A) / per-column
// ones of op(B); k_slice writes the digits as BF16 or FP16 slices (K
// contiguous, padded to a multiple of 32); operands with short rows take both
// steps in one pass (k_slice7f); the products run in k_split_umma
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
// (every launch covers exactly the tiles of its operands, whatever their sizes;
// an operand with no tile in a launch shares its first tile with the next one
// and is never chosen).  Launch: 0 exponents, 1 slices, 2 one-pass slices.
__device__ __forceinline__ int sl_first(const SliceDesc& d, int launch)
{
    return launch == 0 ? d.t_exp : (launch == 1 ? d.t_sl : d.t_fu);
}
__device__ __forceinline__ int sl_operand(const SliceDesc* D, int nop, int t, int launch)
{
    int lo = 0, hi = nop - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sl_first(D[mid], launch) <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int exp_field(double x)
{
    return (__double2hiint(x) >> 20) & 0x7ff;
}

// Rows of an exponent-pass tile: 128 when rows are contiguous in memory (four
// warps read 1 KiB runs of a column: measured, 256-byte runs of columns 64 KiB
// apart held the pass at a third of the DRAM bandwidth), else 32.
__host__ __device__ __forceinline__ int se_rows(long long sr) { return sr == 1 ? 128 : 32; }
// k range of an exponent-pass tile: 256 with 128-row tiles (so the CTA count,
// and the loads in flight, match the 32-row form), SE_K otherwise
__host__ __device__ __forceinline__ int se_kchunk(long long sr) { return sr == 1 ? 256 : SE_K; }

__global__ void k_slice_exp(const SliceDesc* D, int nop)
{
    const int t = blockIdx.x;
    const SliceDesc d = D[sl_operand(D, nop, t, 0)];
    const int RT = se_rows(d.sr);
    const int ry = (d.rows + RT - 1) / RT;
    const int local = t - d.t_exp;
    const int r0 = (local % ry) * RT;
    const int kb = (local / ry) * se_kchunk(d.sr);
    const int nrows = (d.dynK && d.dyn_rows) ? *d.dynK : d.rows;   // actual sizes
    const int Kact = d.dynK ? *d.dynK : d.K;
    if (r0 >= nrows || kb >= Kact) return;
    const int ke = min(Kact, kb + se_kchunk(d.sr));
    __shared__ int red[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    if (d.sr == 1) {
        // rows contiguous: lane = row; warp ty takes rows 32 (ty & 3) + lane and
        // every other column (phase ty >> 2), sixteen independent loads in flight
        // (the pass is bound by load latency)
        const int r = r0 + 32 * (ty & 3) + tx;
        const int kp = ty >> 2;
        int mx = 0;
        if (d.twin_e) {
            // also the column maxima (the twin's row bounds): every lane runs the
            // loop (rows past the end read as zero) for the warp maxima over its rows
            __shared__ int s_cm[256];
            for (int i = threadIdx.x; i < 256; i += 256) s_cm[i] = 0;
            __syncthreads();
            for (int k = kb + kp; k < ke; k += 32) {
                double v[16];
#pragma unroll
                for (int j = 0; j < 16; j++) v[j] = (r < nrows && k + 2 * j < ke) ? slice_load(d, r, k + 2 * j) : 0.0;
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const int f = exp_field(v[j]);
                    mx = max(mx, f);
                    const int cm = __reduce_max_sync(0xffffffffu, f);
                    if (tx == 0 && cm > 0) atomicMax(&s_cm[k + 2 * j - kb], cm);
                }
            }
            __syncthreads();
            for (int i = threadIdx.x; i < ke - kb; i += 256)
                if (s_cm[i] > 0) atomicMax(d.twin_e + kb + i, s_cm[i] - 1022);
        } else if (r < nrows) {
            for (int k = kb + kp; k < ke; k += 32) {
                double v[16];
#pragma unroll
                for (int j = 0; j < 16; j++) v[j] = (k + 2 * j < ke) ? slice_load(d, r, k + 2 * j) : 0.0;
#pragma unroll
                for (int j = 0; j < 16; j++) mx = max(mx, exp_field(v[j]));
            }
        }
        red[ty][tx] = mx;
        __syncthreads();
        if (ty < 4 && r < nrows) {
            const int m = max(red[ty][tx], red[ty + 4][tx]);
            if (m > 0) atomicMax(d.e + r, m - 1022);
        }
    } else {
        // k contiguous: lane = k, warp ty handles rows ty, ty+8, ty+16, ty+24
        for (int q = 0; q < 4; q++) {
            const int r = r0 + ty + 8 * q;
            int m = 0;
            if (r < nrows)
                for (int k = kb + tx; k < ke; k += 512) {
                    double v[16];
#pragma unroll
                    for (int j = 0; j < 16; j++) v[j] = (k + 32 * j < ke) ? slice_load(d, r, k + 32 * j) : 0.0;
#pragma unroll
                    for (int j = 0; j < 16; j++) m = max(m, exp_field(v[j]));
                }
            m = __reduce_max_sync(0xffffffffu, m);
            if (tx == 0 && r < nrows && m > 0) atomicMax(d.e + r, m - 1022);
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
#define SL_R 128  // rows of a slicing tile (1 KiB runs of a column-major operand's columns)
#define SL_NT 512 // threads of a slicing CTA
#define SL_G 10   // padded group length (doubles)
#define SL_ROW (8 * SL_G + 2)   // +2: row stride 164 words

// The 64 x 64 tile of the operand at (r0, k0) into shared memory, rows of 8
// padded groups of 8 doubles; all 16 loads of a thread are issued before any
// shared-memory store.
__device__ __forceinline__ void slice_tile_load(const SliceDesc& d, double (*T)[SL_ROW], int r0, int k0,
                                                int nrows, int Kact)
{
    const int tid = threadIdx.x;
    double v[SL_R * SL_T / SL_NT];
#pragma unroll
    for (int t = 0; t < SL_R * SL_T / SL_NT; t++) {
        const int idx = tid + SL_NT * t;
        int r, k;
        if (d.sr == 1) { r = idx % SL_R; k = idx / SL_R; } else { k = idx % SL_T; r = idx / SL_T; }
        v[t] = (r0 + r < nrows && k0 + k < Kact) ? slice_load(d, r0 + r, k0 + k) : 0.0;
    }
#pragma unroll
    for (int t = 0; t < SL_R * SL_T / SL_NT; t++) {
        const int idx = tid + SL_NT * t;
        int r, k;
        if (d.sr == 1) { r = idx % SL_R; k = idx / SL_R; } else { k = idx % SL_T; r = idx / SL_T; }
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
__global__ void __launch_bounds__(SL_NT) k_slice(const SliceDesc* D, int nop)
{
    const int t = blockIdx.x;   // flattened (operand, 64-row tile, 64-wide k tile)
    const SliceDesc d = D[sl_operand(D, nop, t, 1)];
    const int ky = (d.Kp + SL_T - 1) / SL_T;
    const int k0 = ((t - d.t_sl) % ky) * SL_T, r0 = ((t - d.t_sl) / ky) * SL_R;
    // actual sizes (device-sized operands: the upper bounds only place the tiles);
    // digits are written up to the actual K rounded to 32, zero past K
    const int nrows = (d.dynK && d.dyn_rows) ? *d.dynK : d.rows;
    const int Kact = d.dynK ? *d.dynK : d.K;
    const int Kpa = d.dynK ? min(d.Kp, max(32, ((Kact + 31) / 32) * 32)) : d.Kp;
    if (k0 >= Kpa || r0 >= nrows) return;
    extern __shared__ __align__(16) double sl_smem[];
    double (*T)[SL_ROW] = (double (*)[SL_ROW])sl_smem;   // SL_R rows
    const int tid = threadIdx.x;
    slice_tile_load(d, T, r0, k0, nrows, Kact);
    __syncthreads();
    const int bs = d.beta * d.s;
    const unsigned mask = (1u << d.beta) - 1u;
#pragma unroll
    for (int i = 0; i < (SL_R * SL_T / 8) / SL_NT; i++) {
        const int u = tid + SL_NT * i;
        const int r = u / (SL_T / 8), kg = u % (SL_T / 8);
        const int row = r0 + r, kk = k0 + kg * 8;
        if (row >= nrows || kk >= Kpa) continue;
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
// The S slices of 8 consecutive entries src[0..7] (in shared memory, 16-byte
// aligned) of a row with exponent bound e: slice p's 8 values go to dst + p * pstep
// with one 16-byte store.
template <int S>
__device__ __forceinline__ void slice7_emit(const double2* src, int e, __nv_bfloat16* dst, size_t pstep)
{
    constexpr int BS = 7 * S;
    // 64 in every base-128 digit below the top one
    unsigned long long B = 0;
#pragma unroll
    for (int j = 0; j < S - 1; j++) B |= 64ull << (7 * j);
    unsigned long long m[8];
    unsigned sgn[4];   // sign bits of the pairs at bits 15 and 31
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
        *(uint4*)dst = make_uint4(w[0], w[1], w[2], w[3]);
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
        *(uint4*)(dst + (size_t)p * pstep) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

template <int S>
__global__ void __launch_bounds__(SL_NT, 2) k_slice7(const SliceDesc* D, int nop)
{
    const int t = blockIdx.x;   // flattened (operand, 64-row tile, 64-wide k tile)
    const SliceDesc d = D[sl_operand(D, nop, t, 1)];
    const int ky = (d.Kp + SL_T - 1) / SL_T;
    const int k0 = ((t - d.t_sl) % ky) * SL_T, r0 = ((t - d.t_sl) / ky) * SL_R;
    // actual sizes (device-sized operands: the upper bounds only place the tiles);
    // digits are written up to the actual K rounded to 32, zero past K
    const int nrows = (d.dynK && d.dyn_rows) ? *d.dynK : d.rows;
    const int Kact = d.dynK ? *d.dynK : d.K;
    const int Kpa = d.dynK ? min(d.Kp, max(32, ((Kact + 31) / 32) * 32)) : d.Kp;
    if (k0 >= Kpa || r0 >= nrows) return;
    extern __shared__ __align__(16) double sl_smem[];
    double (*T)[SL_ROW] = (double (*)[SL_ROW])sl_smem;   // SL_R rows
    const int tid = threadIdx.x;
    slice_tile_load(d, T, r0, k0, nrows, Kact);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < (SL_R * SL_T / 8) / SL_NT; i++) {
        const int u = tid + SL_NT * i;
        const int r = u / (SL_T / 8), kg = u % (SL_T / 8);
        const int row = r0 + r, kk = k0 + kg * 8;
        if (row >= nrows || kk >= Kpa) continue;
        slice7_emit<S>((const double2*)&T[r][kg * SL_G], d.e[row], d.S + (size_t)row * d.Kp + kk,
                       (size_t)d.rows * d.Kp);
    }
}

// One-pass form for operands with short padded rows (Kp <= SF_KMAX: the
// products of Algorithm 3, whose k ranges are a leaf's columns or a node's
// ranks).  A CTA holds sf_rows(Kp) whole rows (at most SF_ELEMS entries) in
// shared memory (Kp / 8 groups of 8 doubles per row, each padded to 10 as in
// k_slice7), takes each row's exponent bound from the integer maxima of the
// exponent fields, stores it for the product and writes the digits: each operand
// entry is read from memory once, and the exponent launch is not needed.
// Addresses come from a per-tile table of column pointers and row strides (the
// gather, the second term and the layout resolved once per column), so a load
// costs a table read and one multiply-add.  Rows-contiguous operands (sr == 1)
// are read with lanes along rows, each warp keeping one row group, so every
// thread's 16 entries lie in one row and the exponent maxima are taken in
// registers during the load; the others are read with lanes along k and their
// maxima taken from shared memory.  Measured on a 131072 x 188 gathered
// column-major operand: 3.0 TB/s with per-entry address arithmetic, 4.3 TB/s
// with the table and the in-load maxima (identical digits).
#define SF_ELEMS 8192
#define SF_KMAX 256
// rows of a tile: a power of two from 32 to 256 (whole row groups of 32 lanes)
__host__ __device__ __forceinline__ int sf_rows(int Kp)
{
    const int q = SF_ELEMS / Kp;
    return q >= 256 ? 256 : q >= 128 ? 128 : q >= 64 ? 64 : 32;
}
__host__ __device__ __forceinline__ int sf_rowstride(int Kp) { return (Kp / 8) * SL_G + 2; }
// dynamic shared memory of the largest tile (Kp = 32: 256 rows of 42 doubles)
#define SF_SMEM ((size_t)(SF_ELEMS / 8 * SL_G + 2 * (SF_ELEMS / 32)) * sizeof(double))

template <int S>
__global__ void __launch_bounds__(SL_NT, 2) k_slice7f(const SliceDesc* D, int nop)
{
    const int t = blockIdx.x;   // flattened (operand, row tile)
    const SliceDesc& d = D[sl_operand(D, nop, t, 2)];
    const int Kp = d.Kp;
    const int RT = sf_rows(Kp), G = Kp >> 3, rs = sf_rowstride(Kp);
    const int r0 = (t - d.t_fu) * RT;
    // actual sizes, as in k_slice7
    const int nrows = (d.dynK && d.dyn_rows) ? *d.dynK : d.rows;
    const int Kact = d.dynK ? *d.dynK : d.K;
    const int Kpa = d.dynK ? min(Kp, max(32, ((Kact + 31) / 32) * 32)) : Kp;
    if (r0 >= nrows) return;
    extern __shared__ __align__(16) double sl_smem[];
    __shared__ const double* s_col[SF_KMAX];                // entry (r0, k); null past K
    __shared__ long long s_rst[SF_KMAX];                    // row stride of column k
    __shared__ int s_part[SF_ELEMS / 8 + SF_ELEMS / 256];   // per group, index u + u / 32
    __shared__ int s_e[SF_ELEMS / 32];                      // per row
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const bool rows_contig = d.sr == 1;
    if (tid < Kp) {
        const int k = tid;
        const double* p = nullptr;
        long long rst = 0;
        if (k < Kact) {
            if (k >= d.K1) {
                p = d.X2 + r0 * d.sr2 + (long long)(k - d.K1) * d.sk2;
                rst = d.sr2;
            } else {
                p = d.X + r0 * d.sr + (long long)(d.gk ? d.gk[k] : k) * d.sk;
                rst = d.sr;
            }
        }
        s_col[k] = p;
        s_rst[k] = rst;
    }
    if (tid < RT) s_e[tid] = 0;
    __syncthreads();
    if (rows_contig) {
        // warp w keeps row group g = w mod (RT / 32) (rows 32 g + lane) and takes the
        // columns k = (w + 16 j) / (RT / 32), j < 16: all (row group, column) pairs
        int lg = 0;
        while ((32 << lg) < RT) lg++;
        const int r = 32 * (w & ((1 << lg) - 1)) + lane;
        const bool rok = r0 + r < nrows;
        const int npair = (RT >> 5) * Kp;
        double v[SF_ELEMS / SL_NT];
#pragma unroll
        for (int j = 0; j < SF_ELEMS / SL_NT; j++) {
            const int q = w + (SL_NT / 32) * j;
            const double* p = (q < npair) ? s_col[q >> lg] : nullptr;
            v[j] = (p && rok) ? p[r * s_rst[q >> lg]] : 0.0;
        }
        int mx = 0;
#pragma unroll
        for (int j = 0; j < SF_ELEMS / SL_NT; j++) {
            const int q = w + (SL_NT / 32) * j;
            const int k = q >> lg;
            mx = max(mx, exp_field(v[j]));
            if (q < npair) sl_smem[r * rs + (k >> 3) * SL_G + (k & 7)] = v[j];
        }
        atomicMax(&s_e[r], mx);
    } else {
        // lanes along k: flattened index i = k + Kp r stepped by SL_NT without divisions
        const int nel = RT * Kp;
        const int bq = SL_NT / Kp, aq = SL_NT % Kp;
        double v[SF_ELEMS / SL_NT];
        int a = tid % Kp, b = tid / Kp;
#pragma unroll
        for (int i = 0; i < SF_ELEMS / SL_NT; i++) {
            const double* p = (tid + SL_NT * i < nel) ? s_col[a] : nullptr;
            v[i] = (p && r0 + b < nrows) ? p[b * s_rst[a]] : 0.0;
            a += aq; b += bq;
            if (a >= Kp) { a -= Kp; b++; }
        }
        a = tid % Kp; b = tid / Kp;
#pragma unroll
        for (int i = 0; i < SF_ELEMS / SL_NT; i++) {
            if (tid + SL_NT * i < nel) sl_smem[b * rs + (a >> 3) * SL_G + (a & 7)] = v[i];
            a += aq; b += bq;
            if (a >= Kp) { a -= Kp; b++; }
        }
    }
    __syncthreads();
    const int ng = RT * G;
    if (!rows_contig) {
        // largest exponent field of each group of 8, then of each row
#pragma unroll
        for (int i = 0; i < SF_ELEMS / 8 / SL_NT; i++) {
            const int u = tid + SL_NT * i;
            if (u < ng) {
                const int r = u / G, kg = u - r * G;
                const double2* src = (const double2*)&sl_smem[r * rs + kg * SL_G];
                int mx = 0;
#pragma unroll
                for (int j = 0; j < 4; j++) {
                    const double2 x2 = src[j];
                    mx = max(mx, max(exp_field(x2.x), exp_field(x2.y)));
                }
                s_part[u + (u >> 5)] = mx;
            }
        }
        __syncthreads();
        if (tid < RT) {
            int mx = 0;
            for (int kg = 0; kg < G; kg++) {
                const int u = tid * G + kg;
                mx = max(mx, s_part[u + (u >> 5)]);
            }
            s_e[tid] = mx;
        }
        __syncthreads();
    }
    if (tid < RT) {
        // no normal entry: the bound stays far below any exponent (all digits zero)
        const int mx = s_e[tid];
        const int e = mx > 0 ? mx - 1022 : (int)0xC0C0C0C0;
        s_e[tid] = e;
        if (r0 + tid < nrows) d.e[r0 + tid] = e;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SF_ELEMS / 8 / SL_NT; i++) {
        const int u = tid + SL_NT * i;
        if (u >= ng) continue;
        const int r = u / G, kg = u - r * G;
        const int row = r0 + r, kk = kg * 8;
        if (row >= nrows || kk >= Kpa) continue;
        slice7_emit<S>((const double2*)&sl_smem[r * rs + kg * SL_G], s_e[r], d.S + (size_t)row * d.Kp + kk,
                       (size_t)d.rows * d.Kp);
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

// Byte counts of a prepared launch: descriptors, tensor maps, tile offsets and
// exponents (small), and the slices of every operand (large).
static void split_sizes(const std::vector<GemmDesc>& g, const SplitPrec& pr, size_t* desc_bytes,
                        size_t* slice_bytes)
{
    size_t erows = 0, sb = 0;
    for (const GemmDesc& d : g) {
        const int Kt = d.Kd + d.Kd2;
        const int kp = std::max(32, ((Kt + 31) / 32) * 32);
        sb += al256((size_t)pr.s * d.M * kp * 2) + al256((size_t)pr.s * d.N * kp * 2);
        erows += (size_t)d.M + d.N;
    }
    *desc_bytes = al256(erows * 4) + al256(g.size() * 2 * sizeof(SliceDesc)) +
                  al256(g.size() * sizeof(SplitGemmDesc)) + al256(g.size() * sizeof(int)) +
                  al256(g.size() * 2 * sizeof(CUtensorMap)) + 1024;
    *slice_bytes = sb + 256;
}

// Builds the descriptors of one split-product launch (ng problems) with their
// tensor maps, in device memory at desc (descriptors, exponents) and slices
// (operand slices); the uploads are ordered on st.  Problems with device sizes
// (GemmDesc::dynK) are described by their upper bounds.
static int split_prepare(const std::vector<GemmDesc>& gin, char* desc, char* slices,
                         cudaStream_t st, int kind, int bits, SplitLaunch* L)
{
    const SplitPrec pr = split_prec(kind, bits);
    L->pr = pr;
    L->ng = 0;
    std::vector<GemmDesc> g;
    for (const GemmDesc& d : gin)
        if (d.M > 0 && d.N > 0) g.push_back(d);
    if (g.empty()) return TDEIG_OK;
    std::vector<int> kps(g.size());
    double flops = 0.0, tflops = 0.0, sbytes = 0.0, ebytes = 0.0, fbytes = 0.0;
    const int s = pr.s;
    for (size_t i = 0; i < g.size(); i++) {
        const int Kt = g[i].Kd + g[i].Kd2;
        kps[i] = std::max(32, ((Kt + 31) / 32) * 32);
        flops += 2.0 * g[i].M * g[i].N * Kt;
        tflops += 2.0 * g[i].M * g[i].N * Kt * (s * (s + 1) / 2);
    }
    char* p = desc;
    auto take = [&](size_t n) { char* r = p; p += al256(n); return r; };
    char* q = slices;
    auto take_sl = [&](size_t n) { char* r = q; q += al256(n); return r; };
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
    int tiles = 0;
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
        a.rows = d.M; a.K = d.Kd + d.Kd2; a.Kp = kps[i]; a.s = s; a.beta = pr.beta; a.f16 = pr.f16;
        a.S = (__nv_bfloat16*)take_sl((size_t)s * d.M * kps[i] * 2);
        a.e = ebase + eoff;
        a.dynK = d.dynK;
        a.dyn_rows = 0;
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
        b.rows = d.N; b.K = d.Kd + d.Kd2; b.Kp = kps[i]; b.s = s; b.beta = pr.beta; b.f16 = pr.f16;
        b.S = (__nv_bfloat16*)take_sl((size_t)s * d.N * kps[i] * 2);
        b.e = ebase + eoff;
        b.dynK = d.dynK;
        b.dyn_rows = 1;   // op(B)^T rows are the N columns, N = K in device-sized products
        eoff += d.N;
        sl.push_back(a);
        sl.push_back(b);
        SplitGemmDesc sd;
        memset(&sd, 0, sizeof(sd));
        sd.SA = a.S; sd.SB = b.S; sd.ea = a.e; sd.eb = b.e;
        sd.M = d.M; sd.N = d.N; sd.Kp = kps[i]; sd.s = s; sd.beta = pr.beta;
        sd.C = d.C; sd.ldc = d.ldc; sd.ccol = d.ccol; sd.alpha = d.alpha; sd.betac = d.beta;
        sd.rsplit = d.rsplit; sd.ktop_end = d.ktop_end; sd.kbot_beg = d.kbot_beg;
        sd.chunk = pr.chunk; sd.f16 = pr.f16;
        sd.dynK = d.dynK; sd.dynG = d.dynG;
        if (!encode_slices(&tm[2 * i], a.S, kps[i], d.M, s, UM_BM) ||
            !encode_slices(&tm[2 * i + 1], b.S, kps[i], d.N, s, UM_BN))
            return TDEIG_ECUDA;
        sd.tmA = dtm + 2 * i;
        sd.tmB = dtm + 2 * i + 1;
        sd.tiles_m = td_cdiv(d.M, UM_BM);
        sd.tiles_n = td_cdiv(d.N, UM_BN);
        sd.tile0 = tiles;
        tiles += sd.tiles_m * sd.tiles_n;
        sg.push_back(sd);
    }
    // flattened tile lists of the slicing launches: operands with short rows (7-bit
    // digits, not masked) go to the one-pass kernel, the others to the exponent and
    // slicing kernels.  Algorithmic traffic: every operand element read once by each
    // kernel that reads it, 2 s bytes of slices written per padded element.
    const bool fuse = pr.beta == 7 && !pr.f16;
    auto one_pass = [&](const SliceDesc& o) { return fuse && o.Kp <= SF_KMAX && !o.mask; };
    // transposed twins (Y = A Omega then Z = A^T Omega over the same masked A, as
    // ADC2's sampling issues them): Z's exponents come from Y's exponent pass
    std::vector<char> covered(sl.size(), 0);
    for (size_t i = 0; i + 1 < g.size(); i++) {
        const GemmDesc &y = g[i], &z = g[i + 1];
        SliceDesc &ay = sl[2 * i], &az = sl[2 * i + 2];
        if (!y.transA && z.transA && y.A == z.A && y.lda == z.lda && y.amask && y.amask == z.amask &&
            y.Kd2 == 0 && z.Kd2 == 0 && y.M == y.Kd && z.M == z.Kd && y.M == z.M && !y.dynK && !z.dynK &&
            !y.acol && !one_pass(ay) && !one_pass(az) && !covered[2 * i]) {
            ay.twin_e = az.e;
            covered[2 * i + 2] = 1;
        }
    }
    long long nexp = 0, nsl = 0, nfu = 0;
    for (size_t oi = 0; oi < sl.size(); oi++) {
        SliceDesc& o = sl[oi];
        o.t_exp = (int)nexp;
        o.t_sl = (int)nsl;
        o.t_fu = (int)nfu;
        const double elems = (double)o.rows * o.K;
        const double bytes = 8.0 * elems + 2.0 * s * (double)o.rows * o.Kp;
        if (one_pass(o)) {
            nfu += td_cdiv(o.rows, sf_rows(o.Kp));
            fbytes += bytes;
        } else {
            if (!covered[oi]) {
                nexp += (long long)td_cdiv(o.rows, se_rows(o.sr)) * td_cdiv(o.K, se_kchunk(o.sr));
                ebytes += 8.0 * elems;
            }
            nsl += (long long)td_cdiv(o.Kp, SL_T) * td_cdiv(o.rows, SL_R);
            sbytes += bytes;
        }
    }
    if (nexp >= (1ll << 31) || nsl >= (1ll << 31) || nfu >= (1ll << 31)) return TDEIG_EINVAL;
    std::vector<int> t0(sg.size());
    for (size_t i = 0; i < sg.size(); i++) t0[i] = sg[i].tile0;
    if (cudaMemcpyAsync(dtm, tm.data(), tm.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(dt0, t0.data(), t0.size() * sizeof(int), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(dsl, sl.data(), sl.size() * sizeof(SliceDesc), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(dsg, sg.data(), sg.size() * sizeof(SplitGemmDesc), cudaMemcpyHostToDevice, st) !=
            cudaSuccess)
        return TDEIG_ECUDA;
    // the host vectors are pageable: the copies are staged before returning
    L->dsl = dsl; L->nop = (int)sl.size(); L->nexp = nexp; L->nsl = nsl; L->nfu = nfu;
    L->dsg = dsg; L->dt0 = dt0; L->ng = (int)sg.size(); L->tiles = tiles;
    L->ebase = ebase; L->erows = erows;
    L->flops = flops; L->tflops = tflops; L->sbytes = sbytes; L->ebytes = ebytes; L->fbytes = fbytes;
    double kbl = 0.0;
    for (size_t i = 0; i < g.size(); i++)
        kbl += (double)sg[i].tiles_m * sg[i].tiles_n * (kps[i] / UM_BK);
    snprintf(L->note, sizeof(L->note), "[%d,%.0f,%d,%d,%.6e]", tiles, kbl, s, (int)g.size(), tflops);
    return TDEIG_OK;
}

template <int S>
static void launch_slice7(bool fused, unsigned grid, size_t smem, const SliceDesc* dsl, int nop, cudaStream_t st)
{
    const void* fn = fused ? (const void*)k_slice7f<S> : (const void*)k_slice7<S>;
    td_smem_attr(fn, smem);
    if (fused) k_slice7f<S><<<grid, SL_NT, smem, st>>>(dsl, nop);
    else k_slice7<S><<<grid, SL_NT, smem, st>>>(dsl, nop);
}

static void launch_slice7_s(int s, bool fused, unsigned grid, size_t smem, const SliceDesc* dsl, int nop,
                            cudaStream_t st)
{
    switch (s) {
    case 1: launch_slice7<1>(fused, grid, smem, dsl, nop, st); break;
    case 2: launch_slice7<2>(fused, grid, smem, dsl, nop, st); break;
    case 3: launch_slice7<3>(fused, grid, smem, dsl, nop, st); break;
    case 4: launch_slice7<4>(fused, grid, smem, dsl, nop, st); break;
    case 5: launch_slice7<5>(fused, grid, smem, dsl, nop, st); break;
    case 6: launch_slice7<6>(fused, grid, smem, dsl, nop, st); break;
    case 7: launch_slice7<7>(fused, grid, smem, dsl, nop, st); break;
    default: launch_slice7<8>(fused, grid, smem, dsl, nop, st); break;
    }
}

// The kernels of a prepared launch: exponents and slices (two passes for long
// rows, one for short ones), then the tensor-core product.
void split_run(const SplitLaunch& L, int* status, cudaStream_t st, int* rc)
{
    *rc = TDEIG_OK;
    if (L.ng == 0) return;
    const SplitPrec& pr = L.pr;
    if (L.nexp > 0) {
        // bounds start far below any exponent; the one-pass kernel writes its rows' own
        if (cudaMemsetAsync(L.ebase, 0xC0, L.erows * 4, st) != cudaSuccess) {
            *rc = TDEIG_ECUDA;
            return;
        }
        td_prof_begin(st);
        k_slice_exp<<<(unsigned)L.nexp, 256, 0, st>>>(L.dsl, L.nop);
        td_prof_end(st, "k_slice_exp");
    }
    if (L.nsl > 0) {
        const unsigned gs = (unsigned)L.nsl;
        const size_t tile_smem = (size_t)SL_R * SL_ROW * sizeof(double);   // 82 KiB: opt-in size
        td_prof_begin(st);
        if (pr.beta == 7 && !pr.f16) {
            launch_slice7_s(pr.s, false, gs, tile_smem, L.dsl, L.nop, st);
        } else {
            td_smem_attr((const void*)k_slice, tile_smem);
            k_slice<<<gs, SL_NT, tile_smem, st>>>(L.dsl, L.nop);
        }
        td_prof_end(st, "k_slice");
    }
    if (L.nfu > 0) {
        td_prof_begin(st);
        launch_slice7_s(pr.s, true, (unsigned)L.nfu, SF_SMEM, L.dsl, L.nop, st);
        td_prof_end(st, "k_slice_fused");
    }
    umma_launch(L.dsg, L.dt0, L.ng, L.tiles, pr.s, pr.nacc, status, st);
    TdCtx& cx = td_ctx();
    // [tiles, k-blocks over all tiles, slices, problems, tensor flops]
    td_prof_note(L.note);
    cx.split_tensor_flops += L.tflops;
    cx.split_slice_bytes += L.sbytes;
    cx.split_exp_bytes += L.ebytes;
    cx.split_fused_bytes += L.fbytes;
    if (cudaGetLastError() != cudaSuccess) *rc = TDEIG_ECUDA;
}

size_t split_launch_bytes(const std::vector<GemmDesc>& g, int kind, int bits, size_t* desc_bytes)
{
    size_t db = 0, sb = 0;
    split_sizes(g, split_prec(kind, bits), &db, &sb);
    if (desc_bytes) *desc_bytes = db;
    return sb;
}

int split_prepare_at(const std::vector<GemmDesc>& g, char* desc, char* slices, cudaStream_t st,
                     int kind, int bits, SplitLaunch* L)
{
    return split_prepare(g, desc, slices, st, kind, bits, L);
}

int split_reserve(SplitWS& ws, size_t bytes, cudaStream_t st)
{
    if (bytes <= ws.cap) return TDEIG_OK;
    cudaStreamSynchronize(st);
    split_free(ws);
    const size_t want = bytes + bytes / 4;
    if (cudaMalloc(&ws.base, want) != cudaSuccess) {
        cudaGetLastError();
        return TDEIG_ENOMEM;
    }
    ws.cap = want;
    return TDEIG_OK;
}

double split_launch_gemm(const std::vector<GemmDesc>& g, SplitWS& ws, cudaStream_t st, int* rc,
                         int* status, int kind, int bits)
{
    *rc = TDEIG_OK;
    size_t db = 0, sb = 0;
    split_sizes(g, split_prec(kind, bits), &db, &sb);
    if ((*rc = split_reserve(ws, al256(db) + sb, st))) return 0.0;
    SplitLaunch L;
    if ((*rc = split_prepare(g, ws.base, ws.base + al256(db), st, kind, bits, &L))) return 0.0;
    split_run(L, status, st, rc);
    return L.ng ? L.flops : 0.0;
}
